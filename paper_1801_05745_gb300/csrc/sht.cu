// Spherical-harmonic analysis of a HEALPix RING map and its angular power
// spectrum (the full-sky C_l of Sec. 3.2, whose covariance over realisations
// Eq. 10-11 estimates):
//   a_lm = (4 pi / N_pix) sum_p map_p Y*_lm(theta_p, phi_p),  0 <= m <= l <= lmax,
//   C_l  = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1),
// evaluated ring by ring, FP64 throughout:
//   k_ring_transform : per ring, F_m = sum_j map_j e^{-i m phi_j}
//                      = e^{-i m phi_0} X_{m mod n}, X the ring's DFT (radix-2
//                      FFT in shared memory for power-of-two rings, direct
//                      DFT otherwise); F stored m-major.
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
constexpr int kLegPPT = 4;             // ring pairs per thread
constexpr int kLegChunkL = 32;         // l values per reduction round

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

// One block per ring.  Shared memory: twiddles w_k = e^{-2 pi i k / n} and the
// ring's values (real, or complex for the FFT).
__global__ void __launch_bounds__(512)
k_ring_transform(const float* __restrict__ map, int32_t N, int32_t lmax, int32_t nrings,
                 double2* __restrict__ F) {
  extern __shared__ __align__(16) double2 sh[];
  const int r = blockIdx.x;
  const Ring g = ring_geom(N, r);
  const int n = g.n;
  double2* w = sh;            // [n]
  double2* x = sh + n;        // [n]
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)n, &sn, &cs);
    w[k] = make_double2(cs, sn);
  }
  const bool fft = is_pow2(n);
  if (fft) {
    // bit-reversed load, then radix-2 decimation-in-time stages
    int bits = 0;
    while ((1 << bits) < n) ++bits;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int rj = __brev(j) >> (32 - bits);
      x[rj] = make_double2((double)map[g.start + j], 0.0);
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
      const int half = len >> 1, step = n / len;
      for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
        const int grp = t / half, pos = t - grp * half;
        const int a = grp * len + pos, b = a + half;
        const double2 tw = w[pos * step];
        const double2 xb = x[b];
        const double2 p = make_double2(tw.x * xb.x - tw.y * xb.y, tw.x * xb.y + tw.y * xb.x);
        const double2 xa = x[a];
        x[a] = make_double2(xa.x + p.x, xa.y + p.y);
        x[b] = make_double2(xa.x - p.x, xa.y - p.y);
      }
      __syncthreads();
    }
  } else {
    double* xr = reinterpret_cast<double*>(x + n / 2 + 1);   // real input after X[0..n/2]
    for (int j = threadIdx.x; j < n; j += blockDim.x) xr[j] = (double)map[g.start + j];
    __syncthreads();
    const int kmax = min(n / 2, lmax);       // X_{n-k} = conj X_k for real input
    double2 acc[4];
    for (int k0 = 0; k0 <= kmax; k0 += 4 * blockDim.x) {
      int kk[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { kk[u] = k0 + u * blockDim.x + threadIdx.x; acc[u] = make_double2(0.0, 0.0); }
      int idx[4] = {0, 0, 0, 0};
      for (int j = 0; j < n; ++j) {
        const double v = xr[j];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const double2 tw = w[idx[u]];
          acc[u].x = fma(v, tw.x, acc[u].x);
          acc[u].y = fma(v, tw.y, acc[u].y);
          idx[u] += kk[u] <= kmax ? kk[u] : 0;
          idx[u] -= idx[u] >= n ? n : 0;
        }
      }
      __syncthreads();                        // all reads of xr done before X is written
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (kk[u] <= kmax) x[kk[u]] = acc[u];
      __syncthreads();
    }
  }
  __syncthreads();
  // F_m = e^{-i m phi_0} X_{m mod n}, m = 0..lmax
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    const int k = m % n;
    double2 X;
    if (fft || k <= n / 2) X = x[k];
    else { X = x[n - k]; X.y = -X.y; }
    double sn, cs;
    sincospi(-(double)m * g.phi0_pi, &sn, &cs);
    F[(size_t)m * nrings + r] = make_double2(cs * X.x - sn * X.y, cs * X.y + sn * X.x);
  }
}

// lambda_mm of every ring pair p (north ring p) for m = 0..lmax, as
// mu * 2^e with |mu| in [2^-500, 1): lambda_00 = 1/sqrt(4 pi),
// lambda_mm = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1,m-1}.
__global__ void k_lmm(int32_t N, int32_t lmax, int32_t npairs, double* __restrict__ mu,
                      int32_t* __restrict__ ex) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const Ring g = ring_geom(N, p);
  double v = 0.28209479177387814347;   // 1 / sqrt(4 pi)
  int e = 0;
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) {
      v *= -sqrt((2.0 * m + 1.0) / (2.0 * m)) * g.s;
      if (fabs(v) < 0x1p-500) { v *= 0x1p500; e -= 500; }
    }
    mu[(size_t)m * npairs + p] = v;
    ex[(size_t)m * npairs + p] = e;
  }
}

__device__ __forceinline__ double warp_sum_dd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Block (m, chunk): each thread owns kLegPPT ring pairs
// p = chunk * kLegThreads * kLegPPT + q * kLegThreads + t.  Pair p is the
// north ring p and the south ring 4N - 2 - p (the equator ring, p = 2N - 1,
// is its own mirror); lambda_lm(-z) = (-1)^(l+m) lambda_lm(z), so the pair
// contributes lambda_lm(z_p) (F_north +- F_south).  A thread adds its pairs'
// contributions before the warp reduction, so the FP64 additions of the
// reduction are spread over kLegPPT pairs.  Output: partial sums (without
// the 4 pi / N_pix factor) part[chunk][idx(l, m)].
__global__ void __launch_bounds__(kLegThreads)
k_legendre(const double2* __restrict__ F, const double* __restrict__ mu,
           const int32_t* __restrict__ ex, int32_t N, int32_t lmax, int32_t nrings,
           int32_t npairs, int64_t nalm, double2* __restrict__ part) {
  __shared__ double ra[kLegChunkL], rb[kLegChunkL];
  __shared__ double2 red[kLegThreads / 32][kLegChunkL];
  // blockIdx.y in [0, lmax/2] handles m = y and (if distinct) m = lmax - y,
  // which balances the work per block
  const int chunk = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pp[kLegPPT];
  bool have[kLegPPT];
  double z[kLegPPT];
#pragma unroll
  for (int q = 0; q < kLegPPT; ++q) {
    pp[q] = chunk * kLegThreads * kLegPPT + q * kLegThreads + threadIdx.x;
    have[q] = pp[q] < npairs;
    z[q] = have[q] ? ring_geom(N, pp[q]).z : 0.0;
  }
  for (int pass = 0; pass < 2; ++pass) {
    const int m = pass == 0 ? (int)blockIdx.y : lmax - (int)blockIdx.y;
    if (pass == 1 && m <= (int)blockIdx.y) break;
    double2 E[kLegPPT], O[kLegPPT];
    double v1[kLegPPT], v2[kLegPPT], scale[kLegPPT];   // lambda_{l-1}, lambda_{l-2} mantissas
    int e[kLegPPT];
#pragma unroll
    for (int q = 0; q < kLegPPT; ++q) {
      E[q] = make_double2(0.0, 0.0);
      O[q] = E[q];
      v1[q] = 0.0;
      v2[q] = 0.0;
      e[q] = -100000;
      if (have[q]) {
        const int p = pp[q];
        const double2 fn = F[(size_t)m * nrings + p];
        const int ps = nrings - 1 - p;
        const double2 fs = ps != p ? F[(size_t)m * nrings + ps] : make_double2(0.0, 0.0);
        E[q] = make_double2(fn.x + fs.x, fn.y + fs.y);
        O[q] = make_double2(fn.x - fs.x, fn.y - fs.y);
        v1[q] = mu[(size_t)m * npairs + p];
        e[q] = ex[(size_t)m * npairs + p];
      }
      // 2^e folded into F while it is a normal number far from underflow;
      // below 2^-960 the pair's terms (< 2^-460 |F|) are dropped
      scale[q] = e[q] > -960 ? ldexp(1.0, e[q]) : 0.0;
      E[q] = make_double2(E[q].x * scale[q], E[q].y * scale[q]);
      O[q] = make_double2(O[q].x * scale[q], O[q].y * scale[q]);
    }
    const double c1 = sqrt(2.0 * m + 3.0);
    const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;   // index of (l = 0, m)
    for (int l0 = m; l0 <= lmax; l0 += kLegChunkL) {
      const int cnt = min(kLegChunkL, lmax + 1 - l0);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int l = l0 + t;
        if (l >= m + 2) {
          const double ll = (double)l, mm = (double)m, l1 = (double)(l - 1);
          ra[t] = sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm));
          rb[t] = sqrt((l1 * l1 - mm * mm) / (4.0 * l1 * l1 - 1.0));
        } else {
          ra[t] = 0.0;
          rb[t] = 0.0;
        }
      }
      __syncthreads();
      for (int t = 0; t < cnt; ++t) {
        const int l = l0 + t;
        const double at = ra[t], bt = rb[t];
        const bool odd = (l + m) & 1;
        double cr = 0.0, ci = 0.0;
#pragma unroll
        for (int q = 0; q < kLegPPT; ++q) {
          double v;
          if (l == m) {
            v = v1[q];
          } else if (l == m + 1) {
            v = c1 * z[q] * v1[q];
            v2[q] = v1[q];
            v1[q] = v;
          } else {
            v = at * (z[q] * v1[q] - bt * v2[q]);
            v2[q] = v1[q];
            v1[q] = v;
          }
          const double2 f = odd ? O[q] : E[q];
          cr = fma(v, f.x, cr);
          ci = fma(v, f.y, ci);
        }
        cr = warp_sum_dd(cr);
        ci = warp_sum_dd(ci);
        if (lane == 0) red[warp][t] = make_double2(cr, ci);
      }
      // keep the mantissas in range: one step grows them by less than
      // a (1 + b) < 2 sqrt(2 l) <= 2^8, so after a check every kLegChunkL
      // (32) steps they stay below 2^(500 + 256)
#pragma unroll
      for (int q = 0; q < kLegPPT; ++q) {
        while (fabs(v1[q]) > 0x1p500 || fabs(v2[q]) > 0x1p500) {
          v1[q] *= 0x1p-500;
          v2[q] *= 0x1p-500;
          e[q] += 500;
          if (scale[q] > 0.0) {            // exact: powers of two on normal numbers
            E[q] = make_double2(E[q].x * 0x1p500, E[q].y * 0x1p500);
            O[q] = make_double2(O[q].x * 0x1p500, O[q].y * 0x1p500);
            scale[q] = ldexp(1.0, e[q]);
          } else if (e[q] > -960) {        // the factor becomes representable
            scale[q] = ldexp(1.0, e[q]);
            const int p = pp[q];
            const double2 fn = F[(size_t)m * nrings + p];
            const int ps = nrings - 1 - p;
            const double2 fs = ps != p ? F[(size_t)m * nrings + ps] : make_double2(0.0, 0.0);
            E[q] = make_double2((fn.x + fs.x) * scale[q], (fn.y + fs.y) * scale[q]);
            O[q] = make_double2((fn.x - fs.x) * scale[q], (fn.y - fs.y) * scale[q]);
          }
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < kLegThreads / 32; ++w) { sr += red[w][t].x; si += red[w][t].y; }
        part[(size_t)chunk * nalm + base + l0 + t] = make_double2(sr, si);
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

__global__ void k_alm2cl(const double2* __restrict__ alm, int32_t lmax, double* __restrict__ cl) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  double s = 0.0;
  for (int m = 0; m <= l; ++m) {
    const double2 a = alm[(size_t)m * (2 * lmax + 1 - m) / 2 + l];
    const double q = a.x * a.x + a.y * a.y;
    s += m == 0 ? q : 2.0 * q;
  }
  cl[l] = s / (2.0 * l + 1.0);
}

// ------------------------------------------------------------ synthesis --
// map_p = sum_l sum_{m>=0} (2 - delta_m0) Re(a_lm Y_lm(theta_p, phi_p)), the
// real field with a_l,-m = (-1)^m conj(a_lm), ring by ring:
//   k_legendre_synth : G_m(ring) = sum_l a_lm lambda_lm(z_ring), per (m, ring
//                      pair) with the even/odd split of the mirror rings;
//   k_ring_synth     : map_j = sum_{|m| <= lmax} G_m e^{i m phi_j}, folding
//                      m onto the ring's n frequencies and an inverse DFT.
__global__ void __launch_bounds__(kLegThreads)
k_legendre_synth(const double2* __restrict__ alm, const double* __restrict__ mu,
                 const int32_t* __restrict__ ex, int32_t N, int32_t lmax, int32_t nrings,
                 int32_t npairs, double2* __restrict__ G) {
  __shared__ double ra[kLegChunkL], rb[kLegChunkL];
  __shared__ double2 as[kLegChunkL];
  const int chunk = blockIdx.x;
  int pp[kLegPPT];
  bool have[kLegPPT];
  double z[kLegPPT];
#pragma unroll
  for (int q = 0; q < kLegPPT; ++q) {
    pp[q] = chunk * kLegThreads * kLegPPT + q * kLegThreads + threadIdx.x;
    have[q] = pp[q] < npairs;
    z[q] = have[q] ? ring_geom(N, pp[q]).z : 0.0;
  }
  for (int pass = 0; pass < 2; ++pass) {
    const int m = pass == 0 ? (int)blockIdx.y : lmax - (int)blockIdx.y;
    if (pass == 1 && m <= (int)blockIdx.y) break;
    double v1[kLegPPT], v2[kLegPPT];
    int e[kLegPPT];
    double2 ge[kLegPPT], go[kLegPPT];     // sums over l + m even / odd, in units of 2^e
#pragma unroll
    for (int q = 0; q < kLegPPT; ++q) {
      v1[q] = have[q] ? mu[(size_t)m * npairs + pp[q]] : 0.0;
      v2[q] = 0.0;
      e[q] = have[q] ? ex[(size_t)m * npairs + pp[q]] : 0;
      ge[q] = make_double2(0.0, 0.0);
      go[q] = ge[q];
    }
    const double c1 = sqrt(2.0 * m + 3.0);
    const size_t base = (size_t)m * (2 * lmax + 1 - m) / 2;
    for (int l0 = m; l0 <= lmax; l0 += kLegChunkL) {
      const int cnt = min(kLegChunkL, lmax + 1 - l0);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int l = l0 + t;
        as[t] = alm[base + l];
        if (l >= m + 2) {
          const double ll = (double)l, mm = (double)m, l1 = (double)(l - 1);
          ra[t] = sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm));
          rb[t] = sqrt((l1 * l1 - mm * mm) / (4.0 * l1 * l1 - 1.0));
        } else {
          ra[t] = 0.0;
          rb[t] = 0.0;
        }
      }
      __syncthreads();
      for (int t = 0; t < cnt; ++t) {
        const int l = l0 + t;
        const double at = ra[t], bt = rb[t];
        const double2 a = as[t];
        const bool odd = (l + m) & 1;
#pragma unroll
        for (int q = 0; q < kLegPPT; ++q) {
          double v;
          if (l == m) {
            v = v1[q];
          } else if (l == m + 1) {
            v = c1 * z[q] * v1[q];
            v2[q] = v1[q];
            v1[q] = v;
          } else {
            v = at * (z[q] * v1[q] - bt * v2[q]);
            v2[q] = v1[q];
            v1[q] = v;
          }
          double2& g = odd ? go[q] : ge[q];
          g.x = fma(v, a.x, g.x);
          g.y = fma(v, a.y, g.y);
        }
      }
      // mantissas back in range (growth per step < 2^8, see k_legendre); the
      // sums so far are rescaled with them (terms 2^-500 below the current
      // scale may underflow: they are negligible)
#pragma unroll
      for (int q = 0; q < kLegPPT; ++q) {
        while (fabs(v1[q]) > 0x1p500 || fabs(v2[q]) > 0x1p500) {
          v1[q] *= 0x1p-500;
          v2[q] *= 0x1p-500;
          ge[q] = make_double2(ge[q].x * 0x1p-500, ge[q].y * 0x1p-500);
          go[q] = make_double2(go[q].x * 0x1p-500, go[q].y * 0x1p-500);
          e[q] += 500;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kLegPPT; ++q) {
      if (!have[q]) continue;
      const double sc = e[q] > -1070 ? ldexp(1.0, e[q]) : 0.0;
      const int p = pp[q], ps = nrings - 1 - p;
      G[(size_t)m * nrings + p] = make_double2((ge[q].x + go[q].x) * sc, (ge[q].y + go[q].y) * sc);
      if (ps != p)
        G[(size_t)m * nrings + ps] = make_double2((ge[q].x - go[q].x) * sc, (ge[q].y - go[q].y) * sc);
    }
  }
}

// One block per ring: H_k = sum over m = k mod n (0 <= m <= lmax) of
// G_m e^{i m phi_0} plus, for the negative frequencies, the conjugates of
// the terms with m = -k mod n (1 <= m <= lmax); then map_j = sum_k H_k
// e^{2 pi i k j / n} (inverse radix-2 FFT for power-of-two rings, direct
// sum otherwise).  Each H_k is summed by one thread in increasing m.
__global__ void __launch_bounds__(512)
k_ring_synth(const double2* __restrict__ G, int32_t N, int32_t lmax, int32_t nrings,
             float* __restrict__ map) {
  extern __shared__ __align__(16) double2 sh[];
  const int r = blockIdx.x;
  const Ring g = ring_geom(N, r);
  const int n = g.n;
  double2* w = sh;            // [n]: e^{+2 pi i k / n}
  double2* H = sh + n;        // [n]
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)k / (double)n, &sn, &cs);
    w[k] = make_double2(cs, sn);
  }
  const bool fft = is_pow2(n);
  int bits = 0;
  while ((1 << bits) < n) ++bits;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double hx = 0.0, hy = 0.0;
    for (int m = k; m <= lmax; m += n) {              // m = k mod n
      const double2 gm = G[(size_t)m * nrings + r];
      double sn, cs;
      sincospi((double)m * g.phi0_pi, &sn, &cs);
      hx += cs * gm.x - sn * gm.y;
      hy += cs * gm.y + sn * gm.x;
    }
    for (int m = (n - k) % n; m <= lmax; m += n) {    // -m = k mod n
      if (m == 0) continue;
      const double2 gm = G[(size_t)m * nrings + r];
      double sn, cs;
      sincospi((double)m * g.phi0_pi, &sn, &cs);
      hx += cs * gm.x - sn * gm.y;                    // conj(G_m e^{i m phi_0})
      hy -= cs * gm.y + sn * gm.x;
    }
    const int dst = fft ? (int)(__brev(k) >> (32 - bits)) : k;
    H[dst] = make_double2(hx, hy);
  }
  __syncthreads();
  if (fft) {
    for (int len = 2; len <= n; len <<= 1) {
      const int half = len >> 1, step = n / len;
      for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
        const int grp = t / half, pos = t - grp * half;
        const int a = grp * len + pos, b = a + half;
        const double2 tw = w[pos * step];
        const double2 xb = H[b];
        const double2 p = make_double2(tw.x * xb.x - tw.y * xb.y, tw.x * xb.y + tw.y * xb.x);
        const double2 xa = H[a];
        H[a] = make_double2(xa.x + p.x, xa.y + p.y);
        H[b] = make_double2(xa.x - p.x, xa.y - p.y);
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) map[g.start + j] = (float)H[j].x;
  } else {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double s = 0.0;
      int idx = 0;
      for (int k = 0; k < n; ++k) {
        const double2 h = H[k], tw = w[idx];
        s = fma(h.x, tw.x, fma(-h.y, tw.y, s));
        idx += j;
        idx -= idx >= n ? n : 0;
      }
      map[g.start + j] = (float)s;
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
  char* ws = (char*)ws_get(c, kSlotSht, fbytes + lbytes + pbytes + 512);
  if (!ws) return UFC_ERR_ALLOC;
  double2* F = reinterpret_cast<double2*>(ws);
  double* mu = reinterpret_cast<double*>(ws + fbytes);
  int32_t* ex = reinterpret_cast<int32_t*>(ws + fbytes + (size_t)(lmax + 1) * npairs * 8);
  char* pp = ws + fbytes + lbytes;
  pp += (16 - (reinterpret_cast<uintptr_t>(pp) & 15)) & 15;
  double2* part = reinterpret_cast<double2*>(pp);
  const int smem = 2 * 4 * nside * (int)sizeof(double2);
  UFC_CUDA(c, cudaFuncSetAttribute(k_ring_transform, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem));
  {
    ProfScope ps_(c, "k_ring_transform");
    k_ring_transform<<<nrings, 512, smem, c->stream>>>(map, nside, lmax, nrings, F);
  }
  {
    ProfScope ps_(c, "k_lmm");
    k_lmm<<<(npairs + 127) / 128, 128, 0, c->stream>>>(nside, lmax, npairs, mu, ex);
  }
  {
    ProfScope ps_(c, "k_legendre");
    dim3 grid(nchunk, lmax / 2 + 1);
    k_legendre<<<grid, kLegThreads, 0, c->stream>>>(F, mu, ex, nside, lmax, nrings, npairs, nalm,
                                                    part);
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
  const int nchunk = (npairs + kLegThreads * kLegPPT - 1) / (kLegThreads * kLegPPT);
  const size_t gbytes = (size_t)(lmax + 1) * nrings * sizeof(double2);
  const size_t lbytes = (size_t)(lmax + 1) * npairs * (sizeof(double) + sizeof(int32_t));
  char* ws = (char*)ws_get(c, kSlotSht, gbytes + lbytes + 512);
  if (!ws) return UFC_ERR_ALLOC;
  double2* Gm = reinterpret_cast<double2*>(ws);
  double* mu = reinterpret_cast<double*>(ws + gbytes);
  int32_t* ex = reinterpret_cast<int32_t*>(ws + gbytes + (size_t)(lmax + 1) * npairs * 8);
  {
    ProfScope ps_(c, "k_lmm");
    k_lmm<<<(npairs + 127) / 128, 128, 0, c->stream>>>(nside, lmax, npairs, mu, ex);
  }
  {
    ProfScope ps_(c, "k_legendre_synth");
    dim3 grid(nchunk, lmax / 2 + 1);
    k_legendre_synth<<<grid, kLegThreads, 0, c->stream>>>(reinterpret_cast<const double2*>(alm), mu,
                                                          ex, nside, lmax, nrings, npairs, Gm);
  }
  const int smem = 2 * 4 * nside * (int)sizeof(double2);
  UFC_CUDA(c, cudaFuncSetAttribute(k_ring_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  {
    ProfScope ps_(c, "k_ring_synth");
    k_ring_synth<<<nrings, 512, smem, c->stream>>>(Gm, nside, lmax, nrings, map);
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
  k_alm2cl<<<(lmax + 256) / 256, 256, 0, c->stream>>>(reinterpret_cast<const double2*>(alm), lmax,
                                                        cl);
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

}  // namespace ufc
