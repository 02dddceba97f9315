// Shell and HEALPix RING pixel of an observer-relative vector, in three
// stages that give one and the same answer:
//
//  exact stage  (FP64): the fixed FP64 procedure that defines the answer.
//  fast stage   (FP32): evaluates the same quantities in FP32 and accepts a
//               decision only when the FP32 value lies farther from the
//               decision edge than a proven bound on |FP32 - exact real|
//               plus the FP64 procedure's own distance from the exact real.
//  refine stage (double-float): the same test with ~2^-44 arithmetic and a
//               band of 2^-30 relative, for what the fast stage left open.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so the FP64 procedure
// runs only for the rare particles both filters leave undecided.
//
// The FP64 procedure (pixelisation of Sec. 2.4, HEALPix RING, with the tie
// rule of this library).  Every step is one IEEE binary64 operation in
// round-to-nearest, in the order written, with no contraction:
//   d      = x + shift                 (shift = fl(fl(i L) - o) per axis)
//   s2     = dx*dx + dy*dy;  r = sqrt(s2 + dz*dz);  r == 0 -> invalid
//   shell  b with chi_b <= r < chi_{b+1}, within the box's shells
//   z      = dz / r
//   t      in [0,4): octant ratio u = min(|dx|,|dy|)/max(|dx|,|dy|),
//            a = atanq(u) (quarter turns), tq = a or 1 - a (swap),
//            t = tq, 2 - tq, 2 + tq, 4 - tq by quadrant (dx < 0, dy < 0
//            tests), then t = t - 4 if t >= 4; dx = dy = 0 gives t = 0
//   atanq(u): u == 1 -> 1/2; else two half-angle steps
//            v = u/(1 + sqrt(1 + u*u)), w = v/(1 + sqrt(1 + v*v)),
//            p = Horner sum of (-1)^k/(2k+1) s^k, k = 10..0, s = w*w,
//            atanq = (w*p) * 0x1.45f306dc9c883p+1 (the double nearest 8/pi)
//   |z| <= 2/3 (the double 2.0/3.0): t1 = N*(0.5 + t), t2 = N*(0.75*z),
//            jp = floor(t1 - t2), jm = floor(t1 + t2),
//            ir = clamp(N + 1 + jp - jm, 1, 2N+1), ks = 1 - (ir & 1),
//            ip = ((jp + jm - N + ks + 1 + 8N) / 2) mod 4N,
//            pix = 2N(N-1) + (ir-1) 4N + ip
//   else:    tp = t - floor(t), omz = s2/(r*(r + |dz|)),
//            tmp = N*sqrt(3*omz), jp = floor(tp*tmp),
//            jm = floor((1 - tp)*tmp), ir = min(jp + jm + 1, N),
//            ip = floor(t*ir) mod 4 ir,
//            pix = 2 ir(ir-1) + ip (z > 0) or 12N^2 - 2 ir(ir+1) + ip
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ufc {

// ============================ exact stage (FP64) ============================

__device__ __forceinline__ double atanq_exact(double u) {
  if (u == 1.0) return 0.5;
  double v = __ddiv_rn(u, __dadd_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(u, u)))));
  double w = __ddiv_rn(v, __dadd_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(v, v)))));
  double s = __dmul_rn(w, w);
  // Maclaurin coefficients (-1)^k/(2k+1), k = 10 .. 0, as correctly rounded
  // doubles (the compiler rounds each quotient once).
  double p = 1.0 / 21.0;
  p = __dadd_rn(__dmul_rn(p, s), -1.0 / 19.0);
  p = __dadd_rn(__dmul_rn(p, s), 1.0 / 17.0);
  p = __dadd_rn(__dmul_rn(p, s), -1.0 / 15.0);
  p = __dadd_rn(__dmul_rn(p, s), 1.0 / 13.0);
  p = __dadd_rn(__dmul_rn(p, s), -1.0 / 11.0);
  p = __dadd_rn(__dmul_rn(p, s), 1.0 / 9.0);
  p = __dadd_rn(__dmul_rn(p, s), -1.0 / 7.0);
  p = __dadd_rn(__dmul_rn(p, s), 1.0 / 5.0);
  p = __dadd_rn(__dmul_rn(p, s), -1.0 / 3.0);
  p = __dadd_rn(__dmul_rn(p, s), 1.0);
  return __dmul_rn(__dmul_rn(w, p), 0x1.45f306dc9c883p+1);
}

__device__ __forceinline__ double azimuth_exact(double dx, double dy) {
  double ax = fabs(dx), ay = fabs(dy);
  if (ax == 0.0 && ay == 0.0) return 0.0;
  double tq = (ay <= ax) ? atanq_exact(__ddiv_rn(ay, ax))
                         : __dsub_rn(1.0, atanq_exact(__ddiv_rn(ax, ay)));
  double t;
  if (dx >= 0.0) t = (dy >= 0.0) ? tq : __dsub_rn(4.0, tq);
  else t = (dy >= 0.0) ? __dsub_rn(2.0, tq) : __dadd_rn(2.0, tq);
  if (t >= 4.0) t = __dsub_rn(t, 4.0);
  return t;
}

// Pixel of (dx,dy,dz) with r > 0 and s2 = dx*dx + dy*dy as above.
__device__ __forceinline__ int32_t pixel_exact(int32_t N, double dx, double dy,
                                               double dz, double s2, double r) {
  const int64_t n = N;
  double z = __ddiv_rn(dz, r);
  double za = fabs(z);
  double t = azimuth_exact(dx, dy);
  if (za <= 2.0 / 3.0) {
    double t1 = __dmul_rn(double(N), __dadd_rn(0.5, t));
    double t2 = __dmul_rn(double(N), __dmul_rn(0.75, z));
    int64_t jp = int64_t(floor(__dsub_rn(t1, t2)));
    int64_t jm = int64_t(floor(__dadd_rn(t1, t2)));
    int64_t ir = n + 1 + jp - jm;
    ir = ir < 1 ? 1 : (ir > 2 * n + 1 ? 2 * n + 1 : ir);
    int64_t ks = 1 - (ir & 1);
    int64_t ip = ((jp + jm - n + ks + 1 + 8 * n) / 2) % (4 * n);
    return int32_t(2 * n * (n - 1) + (ir - 1) * 4 * n + ip);
  }
  double tp = __dsub_rn(t, floor(t));
  double omz = __ddiv_rn(s2, __dmul_rn(r, __dadd_rn(r, fabs(dz))));
  double tmp = __dmul_rn(double(N), __dsqrt_rn(__dmul_rn(3.0, omz)));
  int64_t jp = int64_t(floor(__dmul_rn(tp, tmp)));
  int64_t jm = int64_t(floor(__dmul_rn(__dsub_rn(1.0, tp), tmp)));
  int64_t ir = jp + jm + 1;
  if (ir > n) ir = n;
  int64_t ip = int64_t(floor(__dmul_rn(t, double(ir)))) % (4 * ir);
  if (z > 0.0) return int32_t(2 * ir * (ir - 1) + ip);
  return int32_t(12 * n * n - 2 * ir * (ir + 1) + ip);
}

// Key of one particle image by the FP64 procedure: shell*npix + pix, or
// kKeyOutside / kKeyInvalid.
__device__ __forceinline__ int32_t key_exact(const ShellTable& st, int32_t lo,
                                             int32_t hi, int32_t N, int32_t npix,
                                             float x, float y, float zc,
                                             double shx, double shy, double shz) {
  if (!isfinite(x) || !isfinite(y) || !isfinite(zc)) return kKeyInvalid;
  double dx = __dadd_rn(double(x), shx);
  double dy = __dadd_rn(double(y), shy);
  double dz = __dadd_rn(double(zc), shz);
  double s2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  double r = __dsqrt_rn(__dadd_rn(s2, __dmul_rn(dz, dz)));
  if (r == 0.0) return kKeyInvalid;
  if (!(r >= st.chi64[lo]) || !(r < st.chi64[hi])) return kKeyOutside;
  int32_t b = lo;
  while (!(r < st.chi64[b + 1])) ++b;
  return b * npix + pixel_exact(N, dx, dy, dz, s2, r);
}

// ============================ fast stage (FP32) =============================

// Exact FP32 helpers that avoid the conversion instructions (float->int,
// round-to-integral), which GB300 executes on its narrow FP64 pipe.  Valid
// for |w| < 2^22: adding 1.5 * 2^23 leaves round(w) in the low mantissa bits.
constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr int32_t kMagicBits = 0x4B400000;     // bit pattern of kMagic

// floor(w) as int and as float, |w| < 2^22.
__device__ __forceinline__ int32_t floor_fast(float w, float& fl) {
  const float r = __fadd_rn(w, kMagic);        // round to nearest integer
  const float rf = __fsub_rn(r, kMagic);       // that integer, exactly
  const bool up = rf > w;
  fl = up ? __fsub_rn(rf, 1.0f) : rf;
  return (__float_as_int(r) - kMagicBits) - (up ? 1 : 0);
}
// float(k) for |k| < 2^22.
__device__ __forceinline__ float i2f_fast(int32_t k) {
  return __fsub_rn(__int_as_float(kMagicBits + k), kMagic);
}

// Floor of w when w is farther than a band b from every integer, else marks
// the decision open; dmin >= b + 2^-23.  r = w + 1.5 2^23 rounds w to the
// nearest integer n (every caller's |w| is below N + 1 <= 8193, far below
// 2^22), d = w - n is exact (both are multiples of ulp(w) and |d| <= 1/2),
// floor(w) = n - [d < 0], and the floor is certain when the distance |d| to
// the nearest integer is at least dmin.  NaN opens the decision.
__device__ __forceinline__ int32_t floor_certain_d(float w, float dmin, bool& open) {
  const float r = __fadd_rn(w, kMagic);
  const float n = __fsub_rn(r, kMagic);
  const float d = __fsub_rn(w, n);
  open |= !(fabsf(d) >= dmin);
  return (__float_as_int(r) - kMagicBits) - (d < 0.0f ? 1 : 0);
}

// atan(q) * 2/pi for q in [0, 1] as q * P(q^2), P of degree 8 with
// coefficients from a weighted least-squares fit of this library; Horner in
// FP32 with fused multiply-adds.  Checked over every float q in [0, 1]: the
// result is within 1.37 u (u = 2^-24) of the exact value; the fast-stage band
// budgets 2 u for it.
__device__ __forceinline__ float atanq_poly(float q) {
  const float s = q * q;
  float p = 0x1.99fe2cp-10f;
  p = fmaf(p, s, -0x1.2c6c52p-7f);
  p = fmaf(p, s, 0x1.9eeee2p-6f);
  p = fmaf(p, s, -0x1.794fbcp-5f);
  p = fmaf(p, s, 0x1.11c51ap-4f);
  p = fmaf(p, s, -0x1.714478p-4f);
  p = fmaf(p, s, 0x1.049362p-3f);
  p = fmaf(p, s, -0x1.b296eap-3f);
  p = fmaf(p, s, 0x1.45f304p-1f);
  return q * p;
}

// Azimuth of the fast stage: t = base + sgn * a (exact-real identity of the
// quadrant/octant cases of the FP64 procedure), a in [0, 1/2] quarter turns.
struct Azim { float a, sa; int32_t base; bool sgn_pos; };

__device__ __forceinline__ Azim azimuth_fast(float dx, float dy, const Bands& bd, bool& open) {
  const float ax = fabsf(dx), ay = fabsf(dy);
  open |= fmaxf(ax, ay) < bd.axy_min;
  const bool sw = ay > ax;
  const float q = __fdividef(fminf(ax, ay), fmaxf(ax, ay));   // one division, either octant
  Azim r;
  r.a = atanq_poly(q);                         // quarter turns, [0, 1/2]
  const bool xp = dx >= 0.0f, yp = dy >= 0.0f;
  // (base, sgn): Q0 (0,+)|(1,-)  Q1 (2,-)|(1,+)  Q2 (2,+)|(3,-)  Q3 (4,-)|(3,+),
  // one nibble (base | sgn << 3) per (xp, yp, sw) in a 32-bit table:
  // base = xp ? (yp ? (sw ? 1 : 0) : (sw ? 3 : 4)) : (yp ? (sw ? 1 : 2) : (sw ? 3 : 2)),
  // sgn = (xp == yp) != sw
  const uint32_t idx = (xp ? 4u : 0u) | (yp ? 2u : 0u) | (sw ? 1u : 0u);
  const uint32_t nib = (0x18B4923Au >> (4u * idx)) & 15u;
  r.base = int32_t(nib & 7u);
  r.sgn_pos = nib >= 8u;
  r.sa = r.sgn_pos ? r.a : -r.a;
  return r;
}

// Equatorial-belt pixel (|z| certainly <= 2/3), or kKeyUndecided.
__device__ __forceinline__ int32_t pixel_fast_eq(int32_t N, const Bands& bd, float dx, float dy,
                                                 float z) {
  bool open = false;
  const Azim az = azimuth_fast(dx, dy, bd, open);
  // floor(N(1/2 + t) -+ 0.75 N z) = I0 + floor(N sa (+1/2 if N = 1) -+ 0.75 N z),
  // I0 = N base + N/2 (N even; base when N = 1)
  const float c = fmaf(bd.fN, az.sa, bd.c0);
  const int32_t I0 = N * az.base + bd.nhalf;
  const int32_t jp = I0 + floor_certain_d(fmaf(-bd.n75, z, c), bd.eq_d, open);
  const int32_t jm = I0 + floor_certain_d(fmaf(bd.n75, z, c), bd.eq_d, open);
  const int32_t ir = N + 1 + jp - jm;
  open |= uint32_t(ir - 1) > uint32_t(2 * N);
  const int32_t ks = 1 - (ir & 1);
  const int32_t ip = ((jp + jm - N + ks + 1 + bd.eight_n) >> 1) & (bd.four_n - 1);
  return open ? kKeyUndecided : bd.ring0 + (ir - 1) * bd.four_n + ip;
}

// Polar-cap pixel (|z| certainly > 2/3), or kKeyUndecided.
__device__ __forceinline__ int32_t pixel_fast_cap(int32_t N, const Bands& bd, float dx, float dy,
                                                  float dz, float r2, float rinv, float z) {
  bool open = false;
  const Azim az = azimuth_fast(dx, dy, bd, open);
  const float s2 = fmaf(dx, dx, dy * dy);
  const float r = r2 * rinv;
  const float omz = __fdividef(s2, r * (r + fabsf(dz)));
  const float o3 = 3.0f * omz;
  float tmp = bd.fN * (o3 * rsqrtf(o3));
  if (!(o3 > 0.0f)) { tmp = 0.0f; open = true; }
  const float tp = az.sgn_pos ? az.a : 1.0f - az.a;
  const int32_t jp = floor_certain_d(tp * tmp, bd.cap_d, open);
  const int32_t jm = floor_certain_d((1.0f - tp) * tmp, bd.cap_d, open);
  int32_t ir = jp + jm + 1;
  open |= ir > N;
  ir = ir > N ? N : ir;
  const float fir = i2f_fast(ir);
  const int32_t fl = floor_certain_d(az.sa * fir, fmaf(bd.ip_per_ir, fir, 0x1p-23f), open);
  int32_t ip = az.base * ir + fl;              // in [-ir, 4.5 ir]
  const int32_t m = 4 * ir;
  ip = ip < 0 ? ip + m : (ip >= m ? ip - m : ip);
  const int32_t pix = (z > 0.0f) ? 2 * ir * (ir - 1) + ip : bd.npix - 2 * ir * (ir + 1) + ip;
  return open ? kKeyUndecided : pix;
}

// Pixel by the fast stage, or kKeyUndecided.  (dx,dy,dz) are the FP32
// observer-relative coordinates with |d - d_exact| <= 2u|d| + 2u^2 smax,
// r2 = fmaf(dz,dz,fmaf(dy,dy,dx*dx)) > bands.r2_min.
__device__ __forceinline__ int32_t pixel_fast(int32_t N, const Bands& bd, float dx,
                                              float dy, float dz, float r2) {
  const float rinv = rsqrtf(r2);
  const float z = dz * rinv;
  const float za = fabsf(z);
  if (za <= bd.z_eq) return pixel_fast_eq(N, bd, dx, dy, z);
  if (za > bd.z_cap) return pixel_fast_cap(N, bd, dx, dy, dz, r2, rinv, z);
  return kKeyUndecided;
}

// Shell of r2 within edges [lo, hi] by the fast stage: returns the shell, -1
// for certainly outside, or -2 for undecided.  Bands are ordered and
// disjoint: lo2[e] <= hi2[e] <= lo2[e+1].
__device__ __forceinline__ int32_t shell_fast(const float* lo2, const float* hi2,
                                              int32_t lo, int32_t hi, float r2) {
  if (r2 < lo2[lo]) return -1;                 // certainly below chi_lo
  int32_t a = lo, b = hi + 1;                  // lo2[a] <= r2 < lo2[b] (b = hi+1: +inf)
  while (b - a > 1) {
    int32_t m = (a + b) >> 1;
    if (r2 < lo2[m]) b = m; else a = m;
  }
  if (r2 < hi2[a]) return -2;                  // inside edge a's band
  return (a < hi) ? a : -1;
}

// ======================= refine stage (double-float) ========================
// Unevaluated sums hi + lo of two FP32 numbers (Dekker, Knuth).  Every
// product and sum uses the _rn intrinsics so that no step is contracted.

struct df { float h, l; };

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.h, y.h);
  df t = two_sum(x.l, y.l);
  s.l = __fadd_rn(s.l, t.h);
  s = quick_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.h, -x.l}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.h, y.h);
  p.l = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, p.l));
  return quick_two_sum(p.h, p.l);
}
__device__ __forceinline__ df df_mulf(df x, float y) {
  df p = two_prod(x.h, y);
  p.l = __fmaf_rn(x.l, y, p.l);
  return quick_two_sum(p.h, p.l);
}
// Quotient and root estimates need only be within a few ulp: each is
// followed by a residual computed in double-float and a correction, so the
// result's error is set by the double-float residuals (about 2^-44
// relative) and not by the estimate.  The fast approximate division and
// reciprocal square root (at most 2 ulp at the magnitudes met here: no
// divisor near 2^126) therefore replace the correctly rounded ones.
__device__ __forceinline__ df df_div(df x, df y) {
  float q1 = __fdividef(x.h, y.h);
  df r = df_sub(x, df_mulf(y, q1));
  float q2 = __fdividef(r.h, y.h);
  r = df_sub(r, df_mulf(y, q2));
  float q3 = __fdividef(r.h, y.h);
  df q = quick_two_sum(q1, q2);
  return df_add(q, {q3, 0.0f});
}
__device__ __forceinline__ df df_sqrt(df x) {
  if (!(x.h > 0.0f)) return {0.0f, 0.0f};
  float s = __fmul_rn(x.h, rsqrtf(x.h));     // NaN for +inf: the callers' r > 0 test fails
  df e = df_sub(x, two_prod(s, s));
  float c = __fdividef(e.h, __fmul_rn(2.0f, s));
  return df_add({s, 0.0f}, {c, 0.0f});
}
// Double-float constants folded at compile time (no conversion at run time).
struct dfc { float h, l; };
__host__ __device__ constexpr dfc make_dfc(double v) {
  return dfc{(float)v, (float)(v - (double)(float)v)};
}
__device__ __forceinline__ df to_df(dfc c) { return {c.h, c.l}; }


// Table of the refine stage's arctangent: atan(k/32) in quarter turns for
// k = 0..32, double-float pairs of the FP64 procedure's values (within a few
// units of 2^-53 of the exact ones).  Every block fills its shared-memory
// copy once (then a barrier before the first key_refine).
constexpr int kAtanTab = 33;
__device__ __forceinline__ void fill_atan_table(float2* tab) {
  for (int k = threadIdx.x; k < kAtanTab; k += blockDim.x) {
    const double v = atanq_exact(double(k) * 0.03125);
    const float h = __double2float_rn(v);
    tab[k] = make_float2(h, __double2float_rn(__dsub_rn(v, double(h))));
  }
}

// atan(u) in quarter turns for u in [0,1] by table reduction: c = k/32 the
// table point nearest u, atan(u) = atan(c) + atan(t) with
// t = (u - c)/(1 + u c), |t| <= 1/64, and atan(t)/t = 1 - s/3 + s^2/5 -
// s^3/7 + ... (s = t^2 <= 2^-12): the omitted terms lie below 2^-50, the
// s^2 and s^3 terms are taken in FP32 (their rounding, times s, below
// 2^-49) and the rest in double-float, so the result keeps the refine
// stage's 2^-44-level error.  (A NaN u gives k = 0 and a NaN result.)
__device__ __forceinline__ df atanq_df(df u, const float2* tab) {
  if (u.h == 1.0f && u.l == 0.0f) return {0.5f, 0.0f};
  int k = __float2int_rn(__fmul_rn(u.h, 32.0f));
  k = k < 0 ? 0 : (k > kAtanTab - 1 ? kAtanTab - 1 : k);
  const float c = __fmul_rn(float(k), 0.03125f);           // exact
  const df t = df_div(df_add(u, {-c, 0.0f}), df_add({1.0f, 0.0f}, df_mulf(u, c)));
  const df s = df_mul(t, t);
  const float tail = __fmul_rn(s.h, __fmaf_rn(s.h, -1.0f / 7.0f, 0.2f));   // s/5 - s^2/7
  constexpr dfc c3 = make_dfc(-1.0 / 3.0);
  const df p = df_add({1.0f, 0.0f}, df_mul(s, df_add(to_df(c3), {tail, 0.0f})));
  constexpr dfc k2pi = make_dfc(0x1.45f306dc9c883p-1);    // 2/pi
  const float2 a0 = tab[k];
  return df_add({a0.x, a0.y}, df_mul(df_mul(t, p), to_df(k2pi)));
}

// Floor of v when v is farther than band from every integer.
__device__ __forceinline__ int32_t floor_df_certain(df v, float band, bool& open) {
  float f;
  int32_t k = floor_fast(v.h, f);
  float rem = __fadd_rn(__fsub_rn(v.h, f), v.l);
  if (rem < 0.0f) { k -= 1; rem += 1.0f; }
  if (rem >= 1.0f) { k += 1; rem -= 1.0f; }
  open |= !(rem >= band) || !(rem < 1.0f - band) || !(fabsf(v.h) < 4194304.0f);
  return k;
}

// Relative band of the refine stage: every refined quantity is within
// 2^-30 (relative) of the exact real value and of the FP64 procedure's value
// (the double-float operations are accurate to about 2^-44 each).
constexpr float kRefineRel = 9.3132257e-10f;   // 2^-30

// Key of one particle image by the refine stage: shell*npix + pix,
// kKeyOutside, or kKeyUndecided.  d = x + (shf + shlo) per axis; atab is
// the block's copy of the arctangent table (fill_atan_table).
// (chih, chil: the shell edges as double-float, ShellTable's arrays or a
// shared-memory copy of them, which lane-divergent indexing favours)
__device__ __forceinline__ int32_t key_refine(const float* chih, const float* chil,
                                              const float2* atab, int32_t lo,
                                              int32_t hi, int32_t N, int32_t npix,
                                              float x, float y, float zc,
                                              float shx, float shy, float shz,
                                              float lx, float ly, float lz) {
  df dx = df_add(two_sum(x, shx), {lx, 0.0f});
  df dy = df_add(two_sum(y, shy), {ly, 0.0f});
  df dz = df_add(two_sum(zc, shz), {lz, 0.0f});
  df s2 = df_add(df_mul(dx, dx), df_mul(dy, dy));
  df r2 = df_add(s2, df_mul(dz, dz));
  df r = df_sqrt(r2);
  if (!(r.h > 0.0f)) return kKeyUndecided;
  // shell: the last edge whose FP32 part is <= r.h by binary search, then the
  // double-float rule from the edge below it.  Edges are >= 3e-6 apart
  // (relative), far more than an FP32 ulp plus the band, so every edge two
  // or more below the candidate is below r beyond the band.
  int32_t cand = lo - 1;
  for (int32_t L = lo, H = hi; L <= H;) {
    const int32_t mid = (L + H) >> 1;
    if (chih[mid] <= r.h) { cand = mid; L = mid + 1; } else { H = mid - 1; }
  }
  const int32_t e0 = cand - 1 > lo ? cand - 1 : lo;
  int32_t b = e0 - 1;                                // lo - 1: below the first edge
  for (int32_t e = e0; e <= hi; ++e) {
    df c = {chih[e], chil[e]};
    df dd = df_sub(r, c);
    float tol = 4.0f * kRefineRel * r.h;
    if (fabsf(dd.h) <= tol) return kKeyUndecided;
    if (dd.h > 0.0f) b = e; else break;
  }
  if (b < lo || b >= hi) return kKeyOutside;
  bool open = false;
  df z = df_div(dz, r);
  df zabs = (z.h < 0.0f) ? df_neg(z) : z;
  constexpr dfc k23 = make_dfc(2.0 / 3.0);
  df zd = df_sub(zabs, to_df(k23));                  // |z| - 2/3
  if (fabsf(zd.h) <= 4.0f * kRefineRel) return kKeyUndecided;
  bool eq = zd.h < 0.0f;
  float ax = fabsf(dx.h), ay = fabsf(dy.h);
  df axd = dx.h < 0.0f ? df_neg(dx) : dx;
  df ayd = dy.h < 0.0f ? df_neg(dy) : dy;
  if (ax == 0.0f || ay == 0.0f) return kKeyUndecided;
  bool sw = ay > ax;
  df q = sw ? df_div(axd, ayd) : df_div(ayd, axd);
  df a = atanq_df(q, atab);
  int32_t base;
  float sgn;
  if (dx.h >= 0.0f) {
    if (dy.h >= 0.0f) { base = sw ? 1 : 0; sgn = sw ? -1.0f : 1.0f; }
    else              { base = sw ? 3 : 4; sgn = sw ? 1.0f : -1.0f; }
  } else {
    if (dy.h >= 0.0f) { base = sw ? 1 : 2; sgn = sw ? 1.0f : -1.0f; }
    else              { base = sw ? 3 : 2; sgn = sw ? -1.0f : 1.0f; }
  }
  df sa = (sgn > 0.0f) ? a : df_neg(a);
  const float fN = i2f_fast(N);
  int32_t pix;
  if (eq) {
    df c = df_mulf(sa, fN);
    if (N == 1) c = df_add(c, {0.5f, 0.0f});
    int32_t I0 = (N == 1) ? base : N * (2 * base + 1) / 2;
    df zz = df_mulf(z, 0.75f * fN);
    float band = kRefineRel * 8.0f * (2.0f * fN + 1.0f);
    int32_t jp = I0 + floor_df_certain(df_sub(c, zz), band, open);
    int32_t jm = I0 + floor_df_certain(df_add(c, zz), band, open);
    int32_t ir = N + 1 + jp - jm;
    open |= ir < 1 || ir > 2 * N + 1;
    int32_t ks = 1 - (ir & 1);
    int32_t ip = ((jp + jm - N + ks + 1 + 8 * N) >> 1) & (4 * N - 1);
    pix = 2 * N * (N - 1) + (ir - 1) * 4 * N + ip;
  } else {
    df den = df_mul(r, df_add(r, dz.h < 0.0f ? df_neg(dz) : dz));
    df omz = df_div(s2, den);
    df tmp = df_mulf(df_sqrt(df_mulf(omz, 3.0f)), fN);
    df tp = (sgn > 0.0f) ? a : df_sub({1.0f, 0.0f}, a);
    float band = kRefineRel * 8.0f * (fN + 1.0f);
    int32_t jp = floor_df_certain(df_mul(tp, tmp), band, open);
    int32_t jm = floor_df_certain(df_mul(df_sub({1.0f, 0.0f}, tp), tmp), band, open);
    int32_t ir = jp + jm + 1;
    open |= ir > N;
    ir = ir > N ? N : ir;
    int32_t fl = floor_df_certain(df_mulf(sa, i2f_fast(ir)), kRefineRel * 8.0f * i2f_fast(ir + 1), open);
    int32_t ip = base * ir + fl;                    // in [-1.5 ir, 4.5 ir]
    const int32_t m = 4 * ir;
    ip = ip < 0 ? ip + m : (ip >= m ? ip - m : ip);
    pix = (z.h > 0.0f) ? 2 * ir * (ir - 1) + ip : 12 * N * N - 2 * ir * (ir + 1) + ip;
  }
  if (open) return kKeyUndecided;
  return b * npix + pix;
}

}  // namespace ufc
