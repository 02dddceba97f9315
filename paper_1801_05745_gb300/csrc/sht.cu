// Spherical-harmonic analysis of a HEALPix RING map and its angular power
// spectrum (the full-sky C_l of Sec. 3.2, whose covariance over realisations
// Eq. 10-11 estimates):
//   a_lm = (4 pi / N_pix) sum_p map_p Y*_lm(theta_p, phi_p),  0 <= m <= l <= lmax,
//   C_l  = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1),
// evaluated ring by ring in FP64, with the long sums and recurrences in
// double-float (pairs of FP32, about 48 bits) on the FP32 pipe:
//   k_root_table     : the 8 Nside unit roots e^{-2 pi i j / (8 Nside)}.
//   k_ring_transform : per ring, F_m = sum_j map_j e^{-i m phi_j}
//                      = e^{-i m phi_0} X_{m mod n}, X the ring's DFT (radix-2
//                      FFT in shared memory in double-float for power-of-two
//                      rings, twiddles and phases from the root table;
//                      radix-4 split and direct DFTs otherwise); F stored
//                      m-major.
//   k_lmm            : lambda_mm(z) of every north/south ring pair for every m,
//                      as mantissa x 2^exponent (no underflow near the poles).
//   k_legendre       : per (m, chunk of ring pairs) the recurrence over l of
//                      the orthonormal Legendre functions (Condon-Shortley
//                      phase), the pair's even/odd combination of F, and a
//                      block reduction over the pairs -> partial a_lm.
//   k_alm_sum        : a_lm = (4 pi / N_pix) sum of the chunk partials.
//   k_alm2cl         : C_l.
// a_lm is stored m-major (index m (2 lmax + 1 - m) / 2 + l) as FP64 (re, im).
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ctx.h"

namespace ufc {

constexpr int kShtMaxNside = 1024;     // shared-memory FFT of the 4 nside-pixel rings
constexpr int kLegThreads = 256;       // threads per k_legendre block
constexpr int kLegPPT = 4;             // ring pairs per thread (analysis)
constexpr int kSynPPT = 2;             // ring pairs per thread (synthesis: 64 registers,
                                       // 32 warps per SM; 4 pairs take 1.4% longer)
constexpr int kLegChunkL = 32;         // l values per reduction round
static_assert(kLegChunkL == 32, "the block reduction gives each degree of a round one lane");

struct Ring {
  int64_t start;   // first pixel
  int32_t n;       // pixels
  double z, s;     // cos and sin of the colatitude
  double phi0_pi;  // azimuth of the first pixel / pi
};

// Ring r (0-based, north to south) of the RING scheme.
__host__ __device__ inline Ring ring_geom(int32_t N, int32_t r) {
  const int64_t npix = 12ll * N * N;
  const int32_t i = r + 1;
  Ring g;
  if (i < N) {
    g.n = 4 * i;
    g.start = 2ll * i * (i - 1);
    const double t = (double)((int64_t)i * i) / (3.0 * (double)((int64_t)N * N));
    g.z = 1.0 - t;
    g.s = sqrt(t * (2.0 - t));
    g.phi0_pi = 1.0 / (4.0 * i);
  } else if (i <= 3 * N) {
    g.n = 4 * N;
    g.start = 2ll * N * (N - 1) + 4ll * N * (i - N);
    g.z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)N);
    g.s = sqrt((1.0 - g.z) * (1.0 + g.z));
    g.phi0_pi = ((i - N + 1) % 2) / (4.0 * N);
  } else {
    const int32_t k = 4 * N - i;
    g.n = 4 * k;
    g.start = npix - 2ll * k * (k + 1);
    const double t = (double)((int64_t)k * k) / (3.0 * (double)((int64_t)N * N));
    g.z = -(1.0 - t);
    g.s = sqrt(t * (2.0 - t));
    g.phi0_pi = 1.0 / (4.0 * k);
  }
  return g;
}

__device__ __forceinline__ bool is_pow2(int v) { return (v & (v - 1)) == 0; }

// Double-float arithmetic on the FP32 pipe (GB300 runs FP64 at 1/64 of the
// FP32 rate): a value is h + l with |l| <= ulp(h)/2, about 48 bits.  Every
// step is a correctly rounded FP32 intrinsic, so that no contraction changes
// the error-free transformations (Dekker/Knuth two-sum, FMA two-product).
struct dfl { float h, l; };
__device__ __forceinline__ dfl df_from_d(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to_d(dfl a) { return (double)a.h + (double)a.l; }
// h + l with |h| >= |l| renormalised (fast two-sum)
__device__ __forceinline__ dfl df_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  return {s, __fadd_rn(l, __fsub_rn(h, s))};
}
// a * b: the exact product of the high parts plus the cross terms
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_norm(p, e);
}
// a + b (two-sum of the high parts)
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return df_norm(s, __fadd_rn(err, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfl df_scale(dfl a, float p2) { return {a.h * p2, a.l * p2}; }  // exact
// acc += a * b, the low part left unnormalised (renormalised by df_add)
__device__ __forceinline__ void df_mac(dfl& acc, dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  const float pe = __fmaf_rn(a.h, b.h, -p);
  const float s = __fadd_rn(acc.h, p);
  const float bb = __fsub_rn(s, acc.h);
  const float se = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float cross = __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(se, __fadd_rn(pe, cross)));
}

// Complex numbers with double-float parts, (re.h, re.l, im.h, im.l) in a float4.
__device__ __forceinline__ float4 cdf_pack(dfl re, dfl im) { return make_float4(re.h, re.l, im.h, im.l); }
// a * b
__device__ __forceinline__ float4 cdf_mul(float4 a, float4 b) {
  const dfl ar{a.x, a.y}, ai{a.z, a.w}, br{b.x, b.y}, bi{b.z, b.w};
  return cdf_pack(df_add(df_mul(ar, br), df_neg(df_mul(ai, bi))),
                  df_add(df_mul(ar, bi), df_mul(ai, br)));
}
__device__ __forceinline__ float4 cdf_add(float4 a, float4 b) {
  return cdf_pack(df_add(dfl{a.x, a.y}, dfl{b.x, b.y}), df_add(dfl{a.z, a.w}, dfl{b.z, b.w}));
}
__device__ __forceinline__ float4 cdf_sub(float4 a, float4 b) {
  return cdf_pack(df_add(dfl{a.x, a.y}, dfl{-b.x, -b.y}), df_add(dfl{a.z, a.w}, dfl{-b.z, -b.w}));
}
__device__ __forceinline__ float4 cdf_conj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }

// Unit roots e^{-2 pi i j / (8N)}, j < 8N, as double-float complex numbers
// (FP64 sincospi, split once).  Every power-of-two ring (n = 4N, or n = 4i
// with i a power of two) has n | 8N: its FFT twiddles are T[k 8N/n] and the
// phase of its first pixel, e^{-i m phi_0} with phi_0 = pi/n, is
// T[m 4N/n mod 8N].
__global__ void k_root_table(int32_t N, float4* __restrict__ T) {
  const int n8 = 8 * N;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n8; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)j / (double)n8, &sn, &cs);
    T[j] = cdf_pack(df_from_d(cs), df_from_d(sn));
  }
}

// One block per ring.  Shared memory: twiddles w_k = e^{-2 pi i k / n} and the
// ring's values (real, or complex for the FFT).
__global__ void __launch_bounds__(512)
k_ring_transform(const float* __restrict__ map, const float4* __restrict__ T, int32_t N,
                 int32_t lmax, int32_t nrings, double2* __restrict__ F) {
  extern __shared__ __align__(16) double2 sh[];
  const int r = blockIdx.x;
  const Ring g = ring_geom(N, r);
  const int n = g.n;
  if (is_pow2(n)) {
    // radix-2 decimation-in-time FFT in double-float on the FP32 pipe
    // (an FP64 instruction costs the FP32 pipe's time for about 64):
    // bit-reversed load, then the stages; twiddles from the root table
    float4* xd = reinterpret_cast<float4*>(sh);   // [n]
    float4* wd = xd + n;                          // [n/2] e^{-2 pi i k / n}
    const int ts = 8 * N / n;
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) wd[k] = T[k * ts];
    int bits = 0;
    while ((1 << bits) < n) ++bits;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int rj = __brev(j) >> (32 - bits);
      xd[rj] = make_float4(map[g.start + j], 0.f, 0.f, 0.f);
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
      const int half = len >> 1, step = n / len;
      for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
        const int grp = t / half, pos = t - grp * half;
        const int a = grp * len + pos, b = a + half;
        const float4 p = cdf_mul(wd[pos * step], xd[b]);
        const float4 xa = xd[a];
        xd[a] = cdf_add(xa, p);
        xd[b] = cdf_sub(xa, p);
      }
      __syncthreads();
    }
    // F_m = e^{-i m phi_0} X_{m mod n} (phi_0 = 0 or pi/n)
    const bool shifted = g.phi0_pi != 0.0;
    const int ps = 4 * N / n;
    for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
      float4 X = xd[m & (n - 1)];
      if (shifted) X = cdf_mul(T[(m * ps) & (8 * N - 1)], X);
      F[(size_t)m * nrings + r] = make_double2(df_to_d(dfl{X.x, X.y}), df_to_d(dfl{X.z, X.w}));
    }
    return;
  }
  // non power-of-two ring (a polar ring, n = 4 i): one radix-4 split,
  // X_k = sum_{r<4} w_n^{rk} Y_r(k mod i) with Y_r(q) = sum_{a<i} x_{4a+r}
  // w_n^{4aq} the length-i DFTs of the four sub-sequences (real input:
  // Y_r(i-q) = conj Y_r(q), so q <= i/2), then k <= min(n/2, lmax) (real
  // input: X_{n-k} = conj X_k).  Double-float on the FP32 pipe; the map
  // values are FP32.  The twiddles w_n^k come from FP64 sincospi for the
  // first quarter k < i only (w_n^{k + q i} = (-i)^q w_n^k), and the phase
  // e^{-i m phi_0} = w_{2n}^m (phi_0 = pi/n) is w_n^{m/2}, times w_{2n} for
  // odd m.
  float4* wf = reinterpret_cast<float4*>(sh);             // [n] w_n^k
  double2* x = sh + n;
  float* xr = reinterpret_cast<float*>(x);                // [n] the ring's values
  const int ni = n / 4, nq = ni / 2 + 1;
  float4* Y = reinterpret_cast<float4*>(x + n / 4 + 1);   // [4][nq] after xr
  float4* Xf = reinterpret_cast<float4*>(x);              // [n/2 + 1], once xr and Y are read
  for (int jj = threadIdx.x; jj < n; jj += blockDim.x) xr[jj] = map[g.start + jj];
  for (int k = threadIdx.x; k < ni; k += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)n, &sn, &cs);
    const dfl c = df_from_d(cs), sv = df_from_d(sn);
    wf[k] = cdf_pack(c, sv);                              // (c, s)
    wf[k + ni] = cdf_pack(sv, dfl{-c.h, -c.l});           // -i (c + i s)
    wf[k + 2 * ni] = cdf_pack(dfl{-c.h, -c.l}, dfl{-sv.h, -sv.l});
    wf[k + 3 * ni] = cdf_pack(dfl{-sv.h, -sv.l}, c);
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 4 * nq; o += blockDim.x) {
    const int r = o / nq, q = o - r * nq;
    const int step = 4 * q;                  // < n since q <= i/2
    dfl ar{0.f, 0.f}, ai{0.f, 0.f};
    int idx = 0;
    for (int a = 0; a < ni; ++a) {
      const dfl v{xr[4 * a + r], 0.f};
      const float4 tw = wf[idx];
      df_mac(ar, v, dfl{tw.x, tw.y});
      df_mac(ai, v, dfl{tw.z, tw.w});
      idx += step;
      idx -= idx >= n ? n : 0;
    }
    ar = df_add(ar, dfl{0.f, 0.f});
    ai = df_add(ai, dfl{0.f, 0.f});
    Y[o] = make_float4(ar.h, ar.l, ai.h, ai.l);
  }
  __syncthreads();
  const int kmax = min(n / 2, lmax);
  float4 out[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = threadIdx.x + u * (int)blockDim.x;
    if (k > kmax) continue;
    int q = k % ni;
    const bool cj = q > ni / 2;
    if (cj) q = ni - q;
    dfl xre{0.f, 0.f}, xim{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 yv = Y[r * nq + q];
      const dfl yr{yv.x, yv.y}, yi = cj ? dfl{-yv.z, -yv.w} : dfl{yv.z, yv.w};
      const float4 tw = wf[(r * k) % n];
      const dfl tr{tw.x, tw.y}, ti{tw.z, tw.w};
      df_mac(xre, tr, yr);                   // Re(w Y)
      df_mac(xre, df_neg(ti), yi);
      df_mac(xim, tr, yi);                   // Im(w Y)
      df_mac(xim, ti, yr);
    }
    out[u] = cdf_pack(df_add(xre, dfl{0.f, 0.f}), df_add(xim, dfl{0.f, 0.f}));
  }
  __syncthreads();                           // xr and Y are read; X overwrites them
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = threadIdx.x + u * (int)blockDim.x;
    if (k <= kmax) Xf[k] = out[u];
  }
  __syncthreads();
  // F_m = e^{-i m phi_0} X_{m mod n}, m = 0..lmax
  float4 h1;                                 // w_{2n} = e^{-i pi / n}
  {
    double sn, cs;
    sincospi(-1.0 / (double)n, &sn, &cs);
    h1 = cdf_pack(df_from_d(cs), df_from_d(sn));
  }
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    const int k = m % n;
    const float4 X = k <= n / 2 ? Xf[k] : cdf_conj(Xf[n - k]);
    float4 ph = wf[(m >> 1) % n];
    if (m & 1) ph = cdf_mul(ph, h1);
    const float4 v = cdf_mul(ph, X);
    F[(size_t)m * nrings + r] = make_double2(df_to_d(dfl{v.x, v.y}), df_to_d(dfl{v.z, v.w}));
  }
}

// lambda_mm of every ring pair p (north ring p) for m = 0..lmax, as
// mu * 2^e: lambda_00 = 1/sqrt(4 pi),
// lambda_mm = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1}.
// Each thread owns one pair and a run of kLmmRun orders m0 = kLmmRun j ..
// m0 + kLmmRun - 1; it starts from
//   lambda_{m0 m0} = lambda_00 C_j sin(theta)^{m0}        (m0 even: no sign),
//   C_j = prod_{k=1}^{m0} sqrt((2k+1)/(2k))               (pair-independent),
// with sin(theta)^{m0} by repeated squaring, everything as (mantissa in
// [1/2, 1), binary exponent) so that nothing underflows, and then steps
// through its run with the recurrence (the stored mantissas are rescaled
// by 2^500 when they fall below 2^-500).  The block forms the factors
// sqrt((2k+1)/(2k)) and C_j in shared memory: the factors in parallel, one
// run's product per thread, then the prefix products in order by one
// thread.
constexpr int kLmmRun = 64;
constexpr int kLmmMaxRuns = 4 * kShtMaxNside / kLmmRun + 1;   // lmax <= 4 nside
static_assert(kLmmRun % 2 == 0, "runs start at even orders");
struct MantExp { double m; int e; };
__device__ __forceinline__ MantExp me_mul(MantExp a, MantExp b) {
  int d;
  const double x = frexp(a.m * b.m, &d);
  return {x, a.e + b.e + d};
}
__global__ void __launch_bounds__(256)
k_lmm(int32_t N, int32_t lmax, int32_t npairs, double* __restrict__ mu, int32_t* __restrict__ ex) {
  __shared__ double cm[kLmmMaxRuns];
  __shared__ int ce[kLmmMaxRuns];
  __shared__ double fk[4 * kShtMaxNside + 1];   // fk[k] = sqrt((2k+1)/(2k)), k >= 1
  const int nrun = lmax / kLmmRun + 1;
  for (int k = 1 + threadIdx.x; k <= lmax; k += blockDim.x) fk[k] = sqrt((2.0 * k + 1.0) / (2.0 * k));
  __syncthreads();
  for (int j = threadIdx.x; j < nrun; j += blockDim.x) {   // run j-1's factors
    double v = 1.0;
    if (j > 0)
      for (int k = kLmmRun * (j - 1) + 1; k <= kLmmRun * j; ++k) v *= fk[k];
    int d;
    cm[j] = frexp(v, &d);
    ce[j] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 1; j < nrun; ++j) {
      const MantExp c = me_mul({cm[j - 1], ce[j - 1]}, {cm[j], ce[j]});
      cm[j] = c.m;
      ce[j] = c.e;
    }
  __syncthreads();
  const int64_t total = (int64_t)npairs * nrun;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int p = int(t % npairs), j = int(t / npairs);
    const Ring g = ring_geom(N, p);
    const int m0 = kLmmRun * j;
    MantExp r{0.5, 1};                          // 1
    MantExp b;
    b.m = frexp(g.s, &b.e);
    for (int k = m0; k; k >>= 1) {              // s^{m0}
      if (k & 1) r = me_mul(r, b);
      b = me_mul(b, b);
    }
    MantExp l00;
    l00.m = frexp(0.28209479177387814347, &l00.e);   // 1 / sqrt(4 pi)
    const MantExp st = me_mul(me_mul(l00, {cm[j], ce[j]}), r);
    double v = st.m;
    int e = st.e;
    const int mend = min(lmax, m0 + kLmmRun - 1);
    for (int m = m0; m <= mend; ++m) {
      if (m > m0) {
        v *= -fk[m] * g.s;
        if (fabs(v) < 0x1p-500) { v *= 0x1p500; e -= 500; }
      }
      mu[(size_t)m * npairs + p] = v;
      ex[(size_t)m * npairs + p] = e;
    }
  }
}

__device__ __forceinline__ double warp_sum_dd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Recurrence coefficients of every (l, m), m-major like a_lm, as
// double-float pairs (a.h, a.l, b.h, b.l):
//   a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)),
//   b_lm = sqrt(((l-1)^2 - m^2) / (4 (l-1)^2 - 1))   for l >= m + 2, else 0.
// Computed once per call in FP64 (block y = m), so that the Legendre kernels
// read them instead of evaluating FP64 divisions and square roots per block.
__global__ void k_leg_coef(int32_t lmax, float4* __restrict__ coef) {
  const int m = blockIdx.y;
  const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
  for (int l = m + blockIdx.x * blockDim.x + threadIdx.x; l <= lmax; l += gridDim.x * blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l >= m + 2) {
      const double ll = (double)l, mm = (double)m, l1 = (double)(l - 1);
      const dfl a = df_from_d(sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm)));
      const dfl b = df_from_d(sqrt((l1 * l1 - mm * mm) / (4.0 * l1 * l1 - 1.0)));
      v = make_float4(a.h, a.l, b.h, b.l);
    }
    coef[base + l] = v;
  }
}

// Block (m, chunk): each thread owns kLegPPT ring pairs
// p = chunk * kLegThreads * kLegPPT + q * kLegThreads + t.  Pair p is the
// north ring p and the south ring 4N - 2 - p (the equator ring, p = 2N - 1,
// is its own mirror); lambda_lm(-z) = (-1)^(l+m) lambda_lm(z), so the pair
// contributes lambda_lm(z_p) (F_north +- F_south).  The recurrence over l
// and the pair sums run in double-float: lambda_lm = v 2^e with the
// mantissa v brought below 2^30 every 4 steps (a step grows it by less
// than a (1 + b) < 2 sqrt(2 l) <= 2^8, so |v| < 2^62 throughout), the
// factor 2^e folded into the pair's F while e > -120 (below, the pair's
// terms are under 2^-58 |F| and are left out until e grows).  Each degree's
// sum over the pairs: a thread's pairs, then groups of 4 lanes (shuffles),
// then the block's 64 group sums in shared memory (8 per warp, then the 8
// warps' partials, so that the whole block takes part), all in double-float
// (FP64 only for the block's result:
// an FP64 instruction costs the FP32 pipe's time for about 64).  Output:
// partial sums (without the 4 pi / N_pix factor) part[chunk][idx(l, m)].
__global__ void __launch_bounds__(kLegThreads)
k_legendre(const double2* __restrict__ F, const double* __restrict__ mu,
           const int32_t* __restrict__ ex, const float4* __restrict__ coef, int32_t N,
           int32_t lmax, int32_t nrings, int32_t npairs, int64_t nalm,
           double2* __restrict__ part) {
  __shared__ dfl ra[kLegChunkL], rb[kLegChunkL];
  // sums of 4 adjacent lanes (re.h, re.l, im.h, im.l): 8 per warp
  __shared__ float4 red[kLegThreads / 4][kLegChunkL];
  __shared__ float4 red2[kLegThreads / 32][kLegChunkL];   // partials of the 8 warps
  // blockIdx.y in [0, lmax/2] handles m = y and (if distinct) m = lmax - y,
  // which balances the work per block
  const int chunk = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pp[kLegPPT];
  bool have[kLegPPT];
  dfl z[kLegPPT];
#pragma unroll
  for (int q = 0; q < kLegPPT; ++q) {
    pp[q] = chunk * kLegThreads * kLegPPT + q * kLegThreads + threadIdx.x;
    have[q] = pp[q] < npairs;
    z[q] = df_from_d(have[q] ? ring_geom(N, pp[q]).z : 0.0);
  }
  // the pair's (F_north +- F_south) 2^e in double-float, or 0 below 2^-120
  auto fold = [&](int q, int m, int e, dfl* Eo, dfl* Oo) {
    if (!have[q] || e <= -120) {
      Eo[0] = Eo[1] = Oo[0] = Oo[1] = dfl{0.f, 0.f};
      return;
    }
    const int p = pp[q];
    const double2 fn = F[(size_t)m * nrings + p];
    const int ps = nrings - 1 - p;
    const double2 fs = ps != p ? F[(size_t)m * nrings + ps] : make_double2(0.0, 0.0);
    const double sc = ldexp(1.0, e);
    Eo[0] = df_from_d((fn.x + fs.x) * sc);
    Eo[1] = df_from_d((fn.y + fs.y) * sc);
    Oo[0] = df_from_d((fn.x - fs.x) * sc);
    Oo[1] = df_from_d((fn.y - fs.y) * sc);
  };
  for (int pass = 0; pass < 2; ++pass) {
    const int m = pass == 0 ? (int)blockIdx.y : lmax - (int)blockIdx.y;
    if (pass == 1 && m <= (int)blockIdx.y) break;
    dfl E[kLegPPT][2], O[kLegPPT][2];
    dfl v1[kLegPPT], v2[kLegPPT];                 // lambda_{l-1}, lambda_{l-2} mantissas
    int e[kLegPPT];
#pragma unroll
    for (int q = 0; q < kLegPPT; ++q) {
      double mant = 0.0;
      int ee = 0;
      if (have[q]) mant = frexp(mu[(size_t)m * npairs + pp[q]], &ee);   // [0.5, 1) 2^ee
      e[q] = have[q] ? ex[(size_t)m * npairs + pp[q]] + ee : -100000;
      v1[q] = df_from_d(mant);
      v2[q] = dfl{0.f, 0.f};
      fold(q, m, e[q], E[q], O[q]);
    }
    const dfl c1 = df_from_d(sqrt(2.0 * m + 3.0));
    const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;   // index of (l = 0, m)
    for (int l0 = m; l0 <= lmax; l0 += kLegChunkL) {
      const int cnt = min(kLegChunkL, lmax + 1 - l0);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const float4 cv = coef[base + l0 + t];
        ra[t] = dfl{cv.x, cv.y};
        rb[t] = dfl{cv.z, cv.w};
      }
      __syncthreads();
      // two degrees per iteration: (l + m) even, then odd (l0 - m is a
      // multiple of 32), so each half selects its even/odd terms statically
#pragma unroll 2
      for (int t = 0; t < cnt; ++t) {
        const int l = l0 + t;
        const dfl at = ra[t], bt = rb[t];
        const bool odd = (l + m) & 1;
        dfl cr{0.f, 0.f}, ci{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < kLegPPT; ++q) {
          dfl v;
          if (l == m) {
            v = v1[q];
          } else if (l == m + 1) {
            v = df_mul(df_mul(c1, z[q]), v1[q]);
            v2[q] = v1[q];
            v1[q] = v;
          } else {
            v = df_mul(at, df_add(df_mul(z[q], v1[q]), df_neg(df_mul(bt, v2[q]))));
            v2[q] = v1[q];
            v1[q] = v;
          }
          const dfl* f = odd ? O[q] : E[q];
          df_mac(cr, v, f[0]);
          df_mac(ci, v, f[1]);
        }
        // 4 lanes' sums by two shuffle steps; the block step adds the rest
#pragma unroll
        for (int o = 2; o > 0; o >>= 1) {
          const dfl wr{__shfl_down_sync(0xFFFFFFFFu, cr.h, o), __shfl_down_sync(0xFFFFFFFFu, cr.l, o)};
          const dfl wi{__shfl_down_sync(0xFFFFFFFFu, ci.h, o), __shfl_down_sync(0xFFFFFFFFu, ci.l, o)};
          cr = df_add(cr, wr);
          ci = df_add(ci, wi);
        }
        if ((lane & 3) == 0) red[warp * 8 + (lane >> 2)][t] = make_float4(cr.h, cr.l, ci.h, ci.l);
        // keep the mantissas below 2^30 (checked every 4 steps)
        if ((t & 3) == 3) {
#pragma unroll
          for (int q = 0; q < kLegPPT; ++q) {
            while (fabsf(v1[q].h) > 0x1p30f || fabsf(v2[q].h) > 0x1p30f) {
              v1[q] = df_scale(v1[q], 0x1p-30f);
              v2[q] = df_scale(v2[q], 0x1p-30f);
              const bool folded = e[q] > -120;
              e[q] += 30;
              if (folded) {              // exact: powers of two on normal numbers
                E[q][0] = df_scale(E[q][0], 0x1p30f);
                E[q][1] = df_scale(E[q][1], 0x1p30f);
                O[q][0] = df_scale(O[q][0], 0x1p30f);
                O[q][1] = df_scale(O[q][1], 0x1p30f);
              } else {
                fold(q, m, e[q], E[q], O[q]);
              }
            }
          }
        }
      }
      __syncthreads();
      // the 64 group sums of each degree t: warp j adds groups j, j + 8, ...
      // (lane t: conflict-free rows), then 8 partials per degree
      if (lane < cnt) {
        dfl sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll
        for (int w = warp; w < kLegThreads / 4; w += kLegThreads / 32) {
          const float4 v = red[w][lane];
          sr = df_add(sr, dfl{v.x, v.y});
          si = df_add(si, dfl{v.z, v.w});
        }
        red2[warp][lane] = make_float4(sr.h, sr.l, si.h, si.l);
      }
      __syncthreads();
      if (threadIdx.x < cnt) {
        const int t = threadIdx.x;
        dfl sr{0.f, 0.f}, si{0.f, 0.f};
#pragma unroll
        for (int w = 0; w < kLegThreads / 32; ++w) {
          const float4 v = red2[w][t];
          sr = df_add(sr, dfl{v.x, v.y});
          si = df_add(si, dfl{v.z, v.w});
        }
        part[(size_t)chunk * nalm + base + l0 + t] = make_double2(df_to_d(sr), df_to_d(si));
      }
    }
  }
}

__global__ void k_alm_sum(const double2* __restrict__ part, int nchunk, int64_t nalm,
                          double w, double2* __restrict__ alm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
       i += (int64_t)gridDim.x * blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const double2 v = part[(size_t)c * nalm + i];
      sr += v.x;
      si += v.y;
    }
    alm[i] = make_double2(w * sr, w * si);
  }
}

// One warp per degree l: lane k adds the orders m = k, k + 32, ... (their
// loads in flight together), then a fixed shuffle tree.
__global__ void k_alm2cl(const double2* __restrict__ alm, int32_t lmax, double* __restrict__ cl) {
  const int l = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (l > lmax) return;                        // (uniform over the warp)
  double s = 0.0;
  for (int m = lane; m <= l; m += 32) {
    const double2 a = alm[(size_t)m * (2 * lmax + 1 - m) / 2 + l];
    const double q = a.x * a.x + a.y * a.y;
    s += m == 0 ? q : 2.0 * q;
  }
  s = warp_sum_dd(s);
  if (lane == 0) cl[l] = s / (2.0 * l + 1.0);
}

// ------------------------------------------------------------ synthesis --
// map_p = sum_l sum_{m>=0} (2 - delta_m0) Re(a_lm Y_lm(theta_p, phi_p)), the
// real field with a_l,-m = (-1)^m conj(a_lm), ring by ring:
//   k_legendre_synth : G_m(ring) = sum_l a_lm lambda_lm(z_ring), per (m, ring
//                      pair) with the even/odd split of the mirror rings;
//   k_ring_synth     : map_j = sum_{|m| <= lmax} G_m e^{i m phi_j}, folding
//                      m onto the ring's n frequencies and an inverse DFT
//                      (double-float radix-2 FFT with root-table twiddles for
//                      power-of-two rings, radix-4 split otherwise).
__global__ void __launch_bounds__(kLegThreads)
k_legendre_synth(const double2* __restrict__ alm, const double* __restrict__ mu,
                 const int32_t* __restrict__ ex, const float4* __restrict__ coef, int32_t N,
                 int32_t lmax, int32_t nrings, int32_t npairs, double2* __restrict__ G) {
  __shared__ dfl ra[kLegChunkL], rb[kLegChunkL];
  __shared__ dfl as[kLegChunkL][2];
  const int chunk = blockIdx.x;
  int pp[kSynPPT];
  bool have[kSynPPT];
  dfl z[kSynPPT];
#pragma unroll
  for (int q = 0; q < kSynPPT; ++q) {
    pp[q] = chunk * kLegThreads * kSynPPT + q * kLegThreads + threadIdx.x;
    have[q] = pp[q] < npairs;
    z[q] = df_from_d(have[q] ? ring_geom(N, pp[q]).z : 0.0);
  }
  for (int pass = 0; pass < 2; ++pass) {
    const int m = pass == 0 ? (int)blockIdx.y : lmax - (int)blockIdx.y;
    if (pass == 1 && m <= (int)blockIdx.y) break;
    dfl v1[kSynPPT], v2[kSynPPT];
    int e[kSynPPT];
    dfl ge[kSynPPT][2], go[kSynPPT][2];   // sums over l + m even / odd, in units of 2^e
#pragma unroll
    for (int q = 0; q < kSynPPT; ++q) {
      double mant = 0.0;
      int ee = 0;
      if (have[q]) mant = frexp(mu[(size_t)m * npairs + pp[q]], &ee);   // [0.5, 1) 2^ee
      v1[q] = df_from_d(mant);
      v2[q] = dfl{0.f, 0.f};
      e[q] = have[q] ? ex[(size_t)m * npairs + pp[q]] + ee : 0;
      ge[q][0] = ge[q][1] = go[q][0] = go[q][1] = dfl{0.f, 0.f};
    }
    const dfl c1 = df_from_d(sqrt(2.0 * m + 3.0));
    const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
    for (int l0 = m; l0 <= lmax; l0 += kLegChunkL) {
      const int cnt = min(kLegChunkL, lmax + 1 - l0);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int l = l0 + t;
        const double2 a = alm[base + l];
        as[t][0] = df_from_d(a.x);
        as[t][1] = df_from_d(a.y);
        const float4 cv = coef[base + l];
        ra[t] = dfl{cv.x, cv.y};
        rb[t] = dfl{cv.z, cv.w};
      }
      __syncthreads();
      // two degrees per iteration: (l + m) even, then odd (l0 - m is a
      // multiple of 32), so each half selects its even/odd terms statically
#pragma unroll 2
      for (int t = 0; t < cnt; ++t) {
        const int l = l0 + t;
        const dfl at = ra[t], bt = rb[t];
        const dfl ax = as[t][0], ay = as[t][1];
        const bool odd = (l + m) & 1;
#pragma unroll
        for (int q = 0; q < kSynPPT; ++q) {
          dfl v;
          if (l == m) {
            v = v1[q];
          } else if (l == m + 1) {
            v = df_mul(df_mul(c1, z[q]), v1[q]);
            v2[q] = v1[q];
            v1[q] = v;
          } else {
            v = df_mul(at, df_add(df_mul(z[q], v1[q]), df_neg(df_mul(bt, v2[q]))));
            v2[q] = v1[q];
            v1[q] = v;
          }
          dfl* g = odd ? go[q] : ge[q];
          df_mac(g[0], v, ax);
          df_mac(g[1], v, ay);
        }
        // mantissas back below 2^30 every 4 steps (growth per step < 2^8,
        // see k_legendre), so that |v| < 2^62 and the sums stay far from
        // the FP32 range; the sums so far are rescaled with them (terms
        // 2^-30 below the current scale may lose bits: they are negligible)
        if ((t & 3) == 3 || t == cnt - 1) {
#pragma unroll
          for (int q = 0; q < kSynPPT; ++q) {
            while (fabsf(v1[q].h) > 0x1p30f || fabsf(v2[q].h) > 0x1p30f) {
              v1[q] = df_scale(v1[q], 0x1p-30f);
              v2[q] = df_scale(v2[q], 0x1p-30f);
              ge[q][0] = df_scale(ge[q][0], 0x1p-30f);
              ge[q][1] = df_scale(ge[q][1], 0x1p-30f);
              go[q][0] = df_scale(go[q][0], 0x1p-30f);
              go[q][1] = df_scale(go[q][1], 0x1p-30f);
              e[q] += 30;
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kSynPPT; ++q) {
      if (!have[q]) continue;
      const double sc = e[q] > -1070 ? ldexp(1.0, e[q]) : 0.0;
      const double er = df_to_d(ge[q][0]), ei = df_to_d(ge[q][1]);
      const double orr = df_to_d(go[q][0]), oi = df_to_d(go[q][1]);
      const int p = pp[q], ps = nrings - 1 - p;
      G[(size_t)m * nrings + p] = make_double2((er + orr) * sc, (ei + oi) * sc);
      if (ps != p) G[(size_t)m * nrings + ps] = make_double2((er - orr) * sc, (ei - oi) * sc);
    }
  }
}

// One block per ring: H_k = sum over m = k mod n (0 <= m <= lmax) of
// G_m e^{i m phi_0} plus, for the negative frequencies, the conjugates of
// the terms with m = -k mod n (1 <= m <= lmax); then map_j = sum_k H_k
// e^{2 pi i k j / n} (inverse radix-2 FFT for power-of-two rings, direct
// sum otherwise).  Each H_k is summed by one thread in increasing m.
__global__ void __launch_bounds__(512)
k_ring_synth(const double2* __restrict__ G, const float4* __restrict__ T, int32_t N,
             int32_t lmax, int32_t nrings, float* __restrict__ map) {
  extern __shared__ __align__(16) double2 sh[];
  const int r = blockIdx.x;
  const Ring g = ring_geom(N, r);
  const int n = g.n;
  if (is_pow2(n)) {
    // double-float on the FP32 pipe; twiddles e^{+2 pi i k / n} and phases
    // e^{+i m phi_0} (phi_0 = 0 or pi/n) are conjugates of root-table
    // entries; H_k into bit-reversed order, then the inverse FFT stages
    float4* hd = reinterpret_cast<float4*>(sh);   // [n]
    float4* wd = hd + n;                          // [n/2]
    const int ts = 8 * N / n, ps = 4 * N / n;
    const bool shifted = g.phi0_pi != 0.0;
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) wd[k] = cdf_conj(T[k * ts]);
    int bits = 0;
    while ((1 << bits) < n) ++bits;
    auto term = [&](int m) {                    // G_m e^{i m phi_0}
      const double2 gm = G[(size_t)m * nrings + r];
      float4 t = cdf_pack(df_from_d(gm.x), df_from_d(gm.y));
      if (shifted) t = cdf_mul(cdf_conj(T[(m * ps) & (8 * N - 1)]), t);
      return t;
    };
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int m = k; m <= lmax; m += n) h = cdf_add(h, term(m));            // m = k mod n
      for (int m = (n - k) % n; m <= lmax; m += n)                           // -m = k mod n
        if (m != 0) h = cdf_add(h, cdf_conj(term(m)));
      hd[__brev(k) >> (32 - bits)] = h;
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
      const int half = len >> 1, step = n / len;
      for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
        const int grp = t / half, pos = t - grp * half;
        const int a = grp * len + pos, b = a + half;
        const float4 p = cdf_mul(wd[pos * step], hd[b]);
        const float4 xa = hd[a];
        hd[a] = cdf_add(xa, p);
        hd[b] = cdf_sub(xa, p);
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) map[g.start + j] = __fadd_rn(hd[j].x, hd[j].y);
    return;
  }
  {
    // non power-of-two ring (polar, n = 4 i), from the Hermitian half
    // (H_{n-k} = conj H_k, the map being real) with one radix-4 split:
    // map_{4a+r} = Re sum_{q<i} Z_r(q) w^{4aq}, Z_r(q) = sum_{t<4} H_{q+it}
    // w^{r(q+it)}, and Z_r(i-q) = conj Z_r(q), so
    // map_{4a+r} = Re Z_r(0) + 2 sum_{0<q<i/2} Re(Z_r(q) w^{4aq})
    //              + [i even] (-1)^a Re Z_r(i/2).
    // Double-float on the FP32 pipe.  The twiddles w^k = e^{+2 pi i k / n}
    // come from FP64 sincospi for k < i only (w^{k + q i} = i^q w^k); the
    // phases e^{+i m phi_0} = e^{+i pi m / n} are w^{m/2}, times e^{+i pi / n}
    // for odd m.
    float4* wf = reinterpret_cast<float4*>(sh);   // [n] (re.h, re.l, im.h, im.l)
    float4* hf = wf + n;                          // [n/2 + 1]
    const int ni = n / 4, nq = ni / 2 + 1, half = n / 2;
    float4* Z = hf + half + 1;                    // [4][nq]
    for (int k = threadIdx.x; k < ni; k += blockDim.x) {
      double sn, cs;
      sincospi(2.0 * (double)k / (double)n, &sn, &cs);
      const dfl c = df_from_d(cs), sv = df_from_d(sn);
      wf[k] = cdf_pack(c, sv);
      wf[k + ni] = cdf_pack(dfl{-sv.h, -sv.l}, c);                    // i (c + i s)
      wf[k + 2 * ni] = cdf_pack(dfl{-c.h, -c.l}, dfl{-sv.h, -sv.l});
      wf[k + 3 * ni] = cdf_pack(sv, dfl{-c.h, -c.l});
    }
    float4 h1;                                    // e^{+i pi / n}
    {
      double sn, cs;
      sincospi(1.0 / (double)n, &sn, &cs);
      h1 = cdf_pack(df_from_d(cs), df_from_d(sn));
    }
    __syncthreads();
    auto term = [&](int m) {                      // G_m e^{i m phi_0}
      const double2 gm = G[(size_t)m * nrings + r];
      float4 ph = wf[(m >> 1) % n];
      if (m & 1) ph = cdf_mul(ph, h1);
      return cdf_mul(ph, cdf_pack(df_from_d(gm.x), df_from_d(gm.y)));
    };
    for (int k = threadIdx.x; k <= half; k += blockDim.x) {
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int m = k; m <= lmax; m += n) h = cdf_add(h, term(m));          // m = k mod n
      for (int m = (n - k) % n; m <= lmax; m += n)                         // -m = k mod n
        if (m != 0) h = cdf_add(h, cdf_conj(term(m)));
      hf[k] = h;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 4 * nq; o += blockDim.x) {
      const int r = o / nq, q = o - r * nq;
      dfl zr{0.f, 0.f}, zi{0.f, 0.f};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int k = q + ni * t;
        const bool cj = k > half;
        const float4 hv = hf[cj ? n - k : k];
        const dfl hr{hv.x, hv.y}, hi = cj ? dfl{-hv.z, -hv.w} : dfl{hv.z, hv.w};
        const float4 tw = wf[(r * k) % n];
        const dfl tr{tw.x, tw.y}, ti{tw.z, tw.w};
        df_mac(zr, tr, hr);                    // Re(H w)
        df_mac(zr, df_neg(ti), hi);
        df_mac(zi, tr, hi);                    // Im(H w)
        df_mac(zi, ti, hr);
      }
      zr = df_add(zr, dfl{0.f, 0.f});
      zi = df_add(zi, dfl{0.f, 0.f});
      Z[o] = make_float4(zr.h, zr.l, zi.h, zi.l);
    }
    __syncthreads();
    const int qe = (ni + 1) / 2;                 // q in [1, qe): the doubled terms
    for (int jj = threadIdx.x; jj < n; jj += blockDim.x) {
      const int a = jj >> 2, r = jj & 3;
      const float4* Zr = Z + r * nq;
      const int step = (4 * a) % n;              // w^{4aq}: index 4 a q mod n
      dfl acc0{0.f, 0.f}, acc1{0.f, 0.f};
      int idx = step;
      int q = 1;
      for (; q + 1 < qe; q += 2) {
        int idx1 = idx + step;
        idx1 -= idx1 >= n ? n : 0;
        const float4 z0 = Zr[q], t0 = wf[idx], z1 = Zr[q + 1], t1 = wf[idx1];
        df_mac(acc0, dfl{z0.x, z0.y}, dfl{t0.x, t0.y});       // Re(Z w)
        df_mac(acc0, dfl{-z0.z, -z0.w}, dfl{t0.z, t0.w});
        df_mac(acc1, dfl{z1.x, z1.y}, dfl{t1.x, t1.y});
        df_mac(acc1, dfl{-z1.z, -z1.w}, dfl{t1.z, t1.w});
        idx = idx1 + step;
        idx -= idx >= n ? n : 0;
      }
      if (q < qe) {
        const float4 z0 = Zr[q], t0 = wf[idx];
        df_mac(acc0, dfl{z0.x, z0.y}, dfl{t0.x, t0.y});
        df_mac(acc0, dfl{-z0.z, -z0.w}, dfl{t0.z, t0.w});
      }
      dfl sum = df_add(acc0, acc1);
      sum = df_add(sum, sum);                    // the conjugate half
      const float4 z0 = Zr[0];
      sum = df_add(sum, dfl{z0.x, z0.y});
      if ((ni & 1) == 0) {                       // the self-conjugate q = i/2
        const float4 zn = Zr[ni / 2];
        sum = df_add(sum, (a & 1) ? dfl{-zn.x, -zn.y} : dfl{zn.x, zn.y});
      }
      map[g.start + jj] = (float)df_to_d(sum);
    }
  }
}

// a_lm b_l with the Gaussian beam b_l = exp(-l(l+1) sigma^2 / 2).
__global__ void k_alm_beam(const double2* __restrict__ in, int32_t lmax, double sigma,
                           double2* __restrict__ out) {
  const int64_t nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
       i += (int64_t)gridDim.x * blockDim.x) {
    // m from the m-major index: block m starts at s(m) = m (2 lmax + 3 - m) / 2
    // (the entry l = m); take the largest m with s(m) <= i
    const double q = 2.0 * lmax + 3.0;
    int m = (int)((q - sqrt(fmax(q * q - 8.0 * (double)i, 0.0))) / 2.0);
    m = m < 0 ? 0 : (m > lmax ? lmax : m);
    while (m > 0 && (int64_t)m * (2 * lmax + 3 - m) / 2 > i) --m;
    while (m < lmax && (int64_t)(m + 1) * (2 * lmax + 2 - m) / 2 <= i) ++m;
    const int l = (int)(i - (int64_t)m * (2 * lmax + 1 - m) / 2);
    const double b = exp(-0.5 * (double)l * (l + 1) * sigma * sigma);
    const double2 a = in[i];
    out[i] = make_double2(a.x * b, a.y * b);
  }
}

// Band powers: out[b] = mean of C_l over l in [lmin + b dl, lmin + (b+1) dl).
__global__ void k_cl_bin(const double* __restrict__ cl, int32_t lmin, int32_t dl, int32_t nbins,
                         double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  double s = 0.0;
  for (int l = lmin + b * dl; l < lmin + (b + 1) * dl; ++l) s += cl[l];
  out[b] = s / dl;
}

// ------------------------------------------------------------------ host --

ufc_status run_map2alm(ufc_ctx* c, const float* map, int nside, int lmax, double* alm_out) {
  if (!map || !alm_out) return set_err(c, UFC_ERR_ARG, "map_dev and alm_dev are required");
  if (nside < 1 || nside > kShtMaxNside || (nside & (nside - 1)))
    return set_err(c, UFC_ERR_UNSUPPORTED, "map2alm needs a power-of-two nside <= %d", kShtMaxNside);
  if (lmax < 0 || lmax > 4 * nside)
    return set_err(c, UFC_ERR_ARG, "lmax must be in [0, 4 nside]");
  if ((reinterpret_cast<uintptr_t>(alm_out) & 15))
    return set_err(c, UFC_ERR_ARG, "alm_dev must be 16-byte aligned");
  const int nrings = 4 * nside - 1, npairs = 2 * nside;
  const int64_t nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  const int nchunk = (npairs + kLegThreads * kLegPPT - 1) / (kLegThreads * kLegPPT);
  const size_t fbytes = (size_t)(lmax + 1) * nrings * sizeof(double2);
  const size_t lbytes = (size_t)(lmax + 1) * npairs * (sizeof(double) + sizeof(int32_t));
  const size_t pbytes = (size_t)nchunk * nalm * sizeof(double2);
  const size_t cbytes = (size_t)nalm * sizeof(float4);
  const size_t tbytes = (size_t)8 * nside * sizeof(float4);
  char* ws = (char*)ws_get(c, kSlotSht, fbytes + lbytes + pbytes + cbytes + tbytes + 512);
  if (!ws) return UFC_ERR_ALLOC;
  double2* F = reinterpret_cast<double2*>(ws);
  double* mu = reinterpret_cast<double*>(ws + fbytes);
  int32_t* ex = reinterpret_cast<int32_t*>(ws + fbytes + (size_t)(lmax + 1) * npairs * 8);
  char* pp = ws + fbytes + lbytes;
  pp += (16 - (reinterpret_cast<uintptr_t>(pp) & 15)) & 15;
  double2* part = reinterpret_cast<double2*>(pp);
  float4* coef = reinterpret_cast<float4*>(pp + pbytes);
  float4* roots = coef + nalm;
  const int smem = 2 * 4 * nside * (int)sizeof(double2);
  UFC_CUDA(c, cudaFuncSetAttribute(k_ring_transform, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem));
  {
    ProfScope ps_(c, "k_root_table");
    k_root_table<<<(8 * nside + 255) / 256, 256, 0, c->stream>>>(nside, roots);
  }
  {
    ProfScope ps_(c, "k_ring_transform");
    k_ring_transform<<<nrings, 512, smem, c->stream>>>(map, roots, nside, lmax, nrings, F);
  }
  {
    ProfScope ps_(c, "k_lmm");
    const int64_t lt = (int64_t)npairs * (lmax / kLmmRun + 1);
    k_lmm<<<(int)std::min<int64_t>((lt + 255) / 256, 8 * c->num_sms), 256, 0, c->stream>>>(
        nside, lmax, npairs, mu, ex);
  }
  {
    ProfScope ps_(c, "k_leg_coef");
    k_leg_coef<<<dim3(4, lmax + 1), 256, 0, c->stream>>>(lmax, coef);
  }
  {
    ProfScope ps_(c, "k_legendre");
    dim3 grid(nchunk, lmax / 2 + 1);
    k_legendre<<<grid, kLegThreads, 0, c->stream>>>(F, mu, ex, coef, nside, lmax, nrings, npairs,
                                                    nalm, part);
  }
  {
    ProfScope ps_(c, "k_alm_sum");
    const double w = 4.0 * M_PI / (12.0 * (double)nside * nside);
    k_alm_sum<<<2 * c->num_sms, 256, 0, c->stream>>>(part, nchunk, nalm, w,
                                                     reinterpret_cast<double2*>(alm_out));
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

ufc_status run_cl_bin(ufc_ctx* c, const double* cl, int lmax, int lmin, int dl, int nbins,
                      double* out) {
  if (!cl || !out) return set_err(c, UFC_ERR_ARG, "cl_dev and out_dev are required");
  if (lmin < 0 || dl < 1 || nbins < 1 || (int64_t)lmin + (int64_t)nbins * dl > (int64_t)lmax + 1)
    return set_err(c, UFC_ERR_ARG, "bins [lmin, lmin + nbins dl) must lie in [0, lmax]");
  ProfScope ps_(c, "k_cl_bin");
  k_cl_bin<<<(nbins + 255) / 256, 256, 0, c->stream>>>(cl, lmin, dl, nbins, out);
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

ufc_status run_alm2map(ufc_ctx* c, const double* alm, int nside, int lmax, float* map) {
  if (!alm || !map) return set_err(c, UFC_ERR_ARG, "alm_dev and map_dev are required");
  if (nside < 1 || nside > kShtMaxNside || (nside & (nside - 1)))
    return set_err(c, UFC_ERR_UNSUPPORTED, "alm2map needs a power-of-two nside <= %d", kShtMaxNside);
  if (lmax < 0 || lmax > 4 * nside) return set_err(c, UFC_ERR_ARG, "lmax must be in [0, 4 nside]");
  if ((reinterpret_cast<uintptr_t>(alm) & 15))
    return set_err(c, UFC_ERR_ARG, "alm_dev must be 16-byte aligned");
  const int nrings = 4 * nside - 1, npairs = 2 * nside;
  const int nchunk = (npairs + kLegThreads * kSynPPT - 1) / (kLegThreads * kSynPPT);
  const size_t gbytes = (size_t)(lmax + 1) * nrings * sizeof(double2);
  const size_t lbytes = (size_t)(lmax + 1) * npairs * (sizeof(double) + sizeof(int32_t));
  const int64_t nalm = (int64_t)(lmax + 1) * (lmax + 2) / 2;
  const size_t cbytes = (size_t)nalm * sizeof(float4);
  const size_t tbytes = (size_t)8 * nside * sizeof(float4);
  char* ws = (char*)ws_get(c, kSlotSht, gbytes + lbytes + cbytes + tbytes + 512);
  if (!ws) return UFC_ERR_ALLOC;
  double2* Gm = reinterpret_cast<double2*>(ws);
  double* mu = reinterpret_cast<double*>(ws + gbytes);
  int32_t* ex = reinterpret_cast<int32_t*>(ws + gbytes + (size_t)(lmax + 1) * npairs * 8);
  char* cp = ws + gbytes + lbytes;
  cp += (16 - (reinterpret_cast<uintptr_t>(cp) & 15)) & 15;
  float4* coef = reinterpret_cast<float4*>(cp);
  float4* roots = coef + nalm;
  {
    ProfScope ps_(c, "k_root_table");
    k_root_table<<<(8 * nside + 255) / 256, 256, 0, c->stream>>>(nside, roots);
  }
  {
    ProfScope ps_(c, "k_leg_coef");
    k_leg_coef<<<dim3(4, lmax + 1), 256, 0, c->stream>>>(lmax, coef);
  }
  {
    ProfScope ps_(c, "k_lmm");
    const int64_t lt = (int64_t)npairs * (lmax / kLmmRun + 1);
    k_lmm<<<(int)std::min<int64_t>((lt + 255) / 256, 8 * c->num_sms), 256, 0, c->stream>>>(
        nside, lmax, npairs, mu, ex);
  }
  {
    ProfScope ps_(c, "k_legendre_synth");
    dim3 grid(nchunk, lmax / 2 + 1);
    k_legendre_synth<<<grid, kLegThreads, 0, c->stream>>>(reinterpret_cast<const double2*>(alm), mu,
                                                          ex, coef, nside, lmax, nrings, npairs, Gm);
  }
  const int smem = 2 * 4 * nside * (int)sizeof(double2);
  UFC_CUDA(c, cudaFuncSetAttribute(k_ring_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  {
    ProfScope ps_(c, "k_ring_synth");
    k_ring_synth<<<nrings, 512, smem, c->stream>>>(Gm, roots, nside, lmax, nrings, map);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

ufc_status run_alm_beam(ufc_ctx* c, const double* in, int lmax, double sigma, double* out) {
  if (!in || !out) return set_err(c, UFC_ERR_ARG, "alm_in_dev and alm_out_dev are required");
  if (lmax < 0 || !(sigma >= 0.0) || !std::isfinite(sigma))
    return set_err(c, UFC_ERR_ARG, "lmax >= 0 and a finite sigma >= 0 are required");
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return set_err(c, UFC_ERR_ARG, "a_lm buffers must be 16-byte aligned");
  ProfScope ps_(c, "k_alm_beam");
  k_alm_beam<<<2 * c->num_sms, 256, 0, c->stream>>>(reinterpret_cast<const double2*>(in), lmax,
                                                    sigma, reinterpret_cast<double2*>(out));
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

ufc_status run_alm2cl(ufc_ctx* c, const double* alm, int lmax, double* cl) {
  if (!alm || !cl) return set_err(c, UFC_ERR_ARG, "alm_dev and cl_dev are required");
  if (lmax < 0) return set_err(c, UFC_ERR_ARG, "lmax must be >= 0");
  if ((reinterpret_cast<uintptr_t>(alm) & 15))
    return set_err(c, UFC_ERR_ARG, "alm_dev must be 16-byte aligned");
  ProfScope ps_(c, "k_alm2cl");
  k_alm2cl<<<(lmax + 8) / 8, 256, 0, c->stream>>>(reinterpret_cast<const double2*>(alm), lmax,
                                                        cl);
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

}  // namespace ufc
