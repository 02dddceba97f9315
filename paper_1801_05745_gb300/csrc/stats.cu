// kappa map (Eq. 6), moments (Eq. 12-13), PDF (Sec. 3.3), adjoint sums, and
// the Welford covariance over realisations (Eq. 10-11).
//
// GB300 runs FP64 at ~1/64 of FP32, so the per-pixel sums over shells are
// carried in double-float (pairs of FP32, ~2^-44 relative) and converted to
// FP64 only per thread or per block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "pixel.cuh"

namespace ufc {

// ------------------------------------------------------------ helpers -----
struct f2 { float h, l; };

__device__ __forceinline__ f2 f2_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2 f2_norm(float h, float l) {
  float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
// acc += (a_h + a_l) * n, n an exactly representable count.
__device__ __forceinline__ void f2_mac(f2& acc, float ah, float al, float n) {
  float ph = __fmul_rn(ah, n);
  float pe = __fmaf_rn(ah, n, -ph);
  f2 s = f2_two_sum(acc.h, ph);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, __fmaf_rn(al, n, pe)));
}
__device__ __forceinline__ f2 f2_add(f2 x, f2 y) {
  f2 s = f2_two_sum(x.h, y.h);
  return f2_norm(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ f2 f2_mul(f2 x, f2 y) {
  float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
  return f2_norm(p, e);
}
__device__ __forceinline__ double f2_to_d(f2 x) { return double(x.h) + double(x.l); }

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}
// Block sum of a double in fixed order (lane order, then warp order).
template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) t += sh[i];
  return t;   // valid in thread 0
}

struct Coef {
  float ah[kMaxShells];
  float al[kMaxShells];
  float ch, cl;        // C as double-float
  int32_t nshell;
  int32_t npix;
};

// ------------------------------------------------- kappa + adjoint sums ---
// kappa_p = sum_b A_b n_bp - C is accumulated in double-float over the
// shells in order.  The adjoint needs per-shell sums S1_b = sum_p e_p n_bp,
// S2_b = sum_p e_p^2 n_bp, T_b = sum_p g_p n_bp, N_b = sum_p n_bp and global
// sums P_k = sum_p e_p^k (k = 1..3), Q = sum_p g_p of the unrounded map e;
// e, e^2 and g are quantised to pairs of integers and multiplied by the
// counts in exact integer arithmetic.
constexpr int kKT = 256;   // threads of the scalar-load kappa kernel

// round(x) as int for |x| < 2^22, and the rounded value as float (the FP32
// magic-number form of pixel.cuh: no conversion instruction, which GB300
// executes on its narrow FP64 pipe)
__device__ __forceinline__ int32_t round_fast(float x, float& xr) {
  const float r = __fadd_rn(x, kMagic);
  xr = __fsub_rn(r, kMagic);
  return __float_as_int(r) - kMagicBits;
}
// 2^s as float for s in [-126, 127]
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((127 + s) << 23); }
// floor(log2(x)) of a normal float x > 0
__device__ __forceinline__ int ilog2f(float x) { return ((__float_as_int(x) >> 23) & 0xFF) - 127; }

// Splits v (double-float, |v| 2^s < 2^22) into two integers with
// v 2^s = hi + lo 2^-22 to within 2^-23: hi = round(v.h 2^s), lo the rounded
// remainder (|remainder| <= 3/4, so |lo| < 2^22).
__device__ __forceinline__ void quant2(f2 v, int s, int& hi, int& lo) {
  const float sc = pow2f(s);
  const float a = __fmul_rn(v.h, sc);
  float ar;
  hi = round_fast(a, ar);
  const float rem = __fadd_rn(__fsub_rn(a, ar), __fmul_rn(v.l, sc));   // a - ar is exact
  float dummy;
  lo = round_fast(__fmul_rn(rem, 4194304.0f), dummy);                  // 2^22
}

// 128-bit two's-complement fixed-point accumulator (integer operations only).
struct I128 { unsigned long long lo; long long hi; };
// acc += v * 2^sh, sh in [-127, 62]; bits below 2^0 of the result are dropped.
__device__ __forceinline__ void i128_add(I128& acc, long long v, int sh) {
  unsigned long long lo;
  long long hi;
  if (sh >= 64) {
    lo = 0ull;
    hi = v << (sh - 64);
  } else if (sh > 0) {
    lo = (unsigned long long)v << sh;
    hi = v >> (64 - sh);
  } else if (sh == 0) {
    lo = (unsigned long long)v;
    hi = v < 0 ? -1ll : 0ll;
  } else if (sh > -64) {
    const long long t = v >> (-sh);
    lo = (unsigned long long)t;
    hi = t < 0 ? -1ll : 0ll;
  } else {
    lo = v < 0 ? ~0ull : 0ull;
    hi = v < 0 ? -1ll : 0ll;
  }
  const unsigned long long nlo = acc.lo + lo;
  acc.hi += hi + (nlo < acc.lo ? 1ll : 0ll);
  acc.lo = nlo;
}
__device__ __forceinline__ double i128_to_d(I128 a, int frac_bits) {
  return ldexp((double)a.hi * 18446744073709551616.0 + (double)a.lo, -frac_bits);
}
// Fractional bits of the adjoint sums S1 (e n), S2 (e^2 n), T (g n); with
// |e|, |g| < 2^14 and |e|^2 < 2^28 every sum fits the 128-bit range.
constexpr int kFrac1 = 72, kFrac2 = 56, kFrac3 = 72;
struct AdjRow { I128 s[3]; long long n; long long pad_; };

// Forward pass with scalar loads, for a kappa buffer that is not 16-byte
// aligned.
__global__ void __launch_bounds__(kKT)
k_kappa_plain(const int32_t* __restrict__ counts, Coef cf, float* __restrict__ kappa,
              double* __restrict__ ksum_part) {
  __shared__ float ah_s[kMaxShells], al_s[kMaxShells];
  __shared__ double red[kKT / 32];
  const int S = cf.nshell;
  for (int i = threadIdx.x; i < S; i += blockDim.x) { ah_s[i] = cf.ah[i]; al_s[i] = cf.al[i]; }
  __syncthreads();
  f2 ks{0.f, 0.f};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < cf.npix; p += gridDim.x * blockDim.x) {
    f2 acc{0.f, 0.f};
#pragma unroll 8
    for (int b = 0; b < S; ++b)
      f2_mac(acc, ah_s[b], al_s[b], float(__ldcs(counts + (size_t)b * cf.npix + p)));
    f2 e = f2_add(f2_norm(acc.h, acc.l), f2{-cf.ch, -cf.cl});
    const float kf = __fadd_rn(e.h, e.l);
    kappa[p] = kf;
    ks = f2_add(ks, f2{kf, 0.f});
  }
  const double t = block_sum_d<kKT>(f2_to_d(ks), red);
  if (threadIdx.x == 0) ksum_part[blockIdx.x] = t;
}

// Forward pass with vector loads: each thread owns 4 adjacent pixels and
// reads every shell row of them as one 16-byte streaming load, 8 rows in
// flight; no staging and no barriers, several blocks per SM.  Needs 16-byte
// aligned counts and kappa (12 nside^2 is a multiple of 4).
constexpr int kKV = 256;
__device__ __forceinline__ float kappa_round(f2 a, f2 mc) {
  const f2 e = f2_add(f2_norm(a.h, a.l), mc);   // e = acc - C (unrounded)
  return __fadd_rn(e.h, e.l);
}
// One block's share of the vector-load forward pass: block vb of a grid of nb
// blocks of kKV threads (every thread of the block calls it); returns the
// block's sum of the FP32 kappa values, valid in thread 0.
__device__ __forceinline__ double kappa_vec_block(const int32_t* __restrict__ counts,
                                                  const float* ah_s, const float* al_s, int S,
                                                  int npix, f2 mc, float* __restrict__ kappa,
                                                  int vb, int nb, double* red) {
  const int ng = npix >> 2;
  const int4* c4 = reinterpret_cast<const int4*>(counts);
  f2 ks{0.f, 0.f};
  for (int g = vb * kKV + threadIdx.x; g < ng; g += nb * kKV) {
    f2 a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
#pragma unroll 8
    for (int b = 0; b < S; ++b) {
      const int4 n = __ldcs(c4 + (size_t)b * ng + g);
      const float h = ah_s[b], l = al_s[b];
      f2_mac(a0, h, l, float(n.x));
      f2_mac(a1, h, l, float(n.y));
      f2_mac(a2, h, l, float(n.z));
      f2_mac(a3, h, l, float(n.w));
    }
    const float4 kv = make_float4(kappa_round(a0, mc), kappa_round(a1, mc), kappa_round(a2, mc),
                                  kappa_round(a3, mc));
    reinterpret_cast<float4*>(kappa)[g] = kv;
    ks = f2_add(ks, f2_add(f2_two_sum(kv.x, kv.y), f2_two_sum(kv.z, kv.w)));
  }
  return block_sum_d<kKV>(f2_to_d(ks), red);
}

__global__ void __launch_bounds__(kKV)
k_kappa_vec(const int32_t* __restrict__ counts, Coef cf, float* __restrict__ kappa,
            double* __restrict__ ksum_part) {
  __shared__ float ah_s[kMaxShells], al_s[kMaxShells];
  __shared__ double red[kKV / 32];
  const int S = cf.nshell;
  for (int i = threadIdx.x; i < S; i += blockDim.x) { ah_s[i] = cf.ah[i]; al_s[i] = cf.al[i]; }
  __syncthreads();
  const double t = kappa_vec_block(counts, ah_s, al_s, S, cf.npix, f2{-cf.ch, -cf.cl}, kappa,
                                   blockIdx.x, gridDim.x, red);
  if (threadIdx.x == 0) ksum_part[blockIdx.x] = t;
}

// ----------------------------------------- subvolume partial sums -----
// Sec. 2.4 processes subvolumes independently and combines their maps; kappa
// is linear in the counts, so a subvolume contributes its partial sum
// e_p = sum_b A_b n_bp (no -C) and the map is kappa_p = (sum over
// subvolumes of e_p) - C.  The partial is accumulated in double-float over
// the shells in order, as the forward pass does, and stored as FP64 (the
// pair's sum), so that the subvolumes' partials add in FP64.
// An FP64 value as a double-float pair (h + l within 2^-48 relative).
__device__ __forceinline__ f2 d_to_f2(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(__dsub_rn(v, (double)h))};
}

__global__ void __launch_bounds__(kKV)
k_kappa_partial(const int32_t* __restrict__ counts, Coef cf, double* __restrict__ part) {
  __shared__ float ah_s[kMaxShells], al_s[kMaxShells];
  const int S = cf.nshell, ng = cf.npix >> 2;
  for (int i = threadIdx.x; i < S; i += blockDim.x) { ah_s[i] = cf.ah[i]; al_s[i] = cf.al[i]; }
  __syncthreads();
  const int4* c4 = reinterpret_cast<const int4*>(counts);
  double2* o2 = reinterpret_cast<double2*>(part);
  for (int g = blockIdx.x * kKV + threadIdx.x; g < ng; g += gridDim.x * kKV) {
    f2 a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
#pragma unroll 8
    for (int b = 0; b < S; ++b) {
      const int4 n = __ldcs(c4 + (size_t)b * ng + g);
      const float h = ah_s[b], l = al_s[b];
      f2_mac(a0, h, l, float(n.x));
      f2_mac(a1, h, l, float(n.y));
      f2_mac(a2, h, l, float(n.z));
      f2_mac(a3, h, l, float(n.w));
    }
    o2[2 * g] = make_double2(f2_to_d(f2_norm(a0.h, a0.l)), f2_to_d(f2_norm(a1.h, a1.l)));
    o2[2 * g + 1] = make_double2(f2_to_d(f2_norm(a2.h, a2.l)), f2_to_d(f2_norm(a3.h, a3.l)));
  }
}

// The FP32 map from the summed partials: kappa_p = (E_p - C) in double-float
// (E_p split into a pair), rounded once to FP32, with the per-block sums of
// the map over the same grid and in the same order as k_kappa_vec, so that
// the moment pass treats it exactly as a map from the counts.
__global__ void __launch_bounds__(kKV)
k_kappa_finish(const double* __restrict__ part, float ch, float cl, int npix,
               float* __restrict__ kappa, double* __restrict__ ksum_part) {
  __shared__ double red[kKV / 32];
  const int ng = npix >> 2;
  const f2 mc{-ch, -cl};
  const double2* p2 = reinterpret_cast<const double2*>(part);
  f2 ks{0.f, 0.f};
  for (int g = blockIdx.x * kKV + threadIdx.x; g < ng; g += gridDim.x * kKV) {
    const double2 d01 = __ldcs(p2 + 2 * g), d23 = __ldcs(p2 + 2 * g + 1);
    const float4 kv = make_float4(kappa_round(d_to_f2(d01.x), mc), kappa_round(d_to_f2(d01.y), mc),
                                  kappa_round(d_to_f2(d23.x), mc), kappa_round(d_to_f2(d23.y), mc));
    reinterpret_cast<float4*>(kappa)[g] = kv;
    ks = f2_add(ks, f2_add(f2_two_sum(kv.x, kv.y), f2_two_sum(kv.z, kv.w)));
  }
  const double t = block_sum_d<kKV>(f2_to_d(ks), red);
  if (threadIdx.x == 0) ksum_part[blockIdx.x] = t;
}

// --------------------------------------------------------- adjoint -----
// One pass (k_adj_main) over tiles of 4 pixels per thread (2560 or 3072
// pixels, the block sizes below), one block per SM.  Phase 1:
// e_p = sum_b A_b n_bp - C unrounded (double-float, the shells in order, as
// the forward pass), e_p^2, the power sums P1..P3 = sum_p e_p^k and
// Q = sum_p g_p, and the tile's maxima of |e|, e^2, |g|.  Each quantity is
// quantised (quant2: two integers, 43 bits relative to the scale) with a
// power-of-two scale from the block's running maximum over the tiles it has
// seen; when a tile raises a maximum, the 64-bit accumulators are first
// flushed at the old scale into the block's 128-bit fixed-point rows, which
// take every flush at its own scale exactly.  Every pixel is therefore
// quantised at least as finely as a single scale from the global maxima
// would.  Phase 2: warp w of NW owns shells w, w + NW, w + 2 NW (of the
// launch's window) and each lane a
// column of the tile's pixels, accumulating q n in 64-bit integers (the
// tile's counts read a second time, mostly from L2).  A bound on the
// accumulated magnitudes (pixels per lane x tile maximum count x 2^22 per
// tile) triggers a flush before any 64-bit sum could overflow.  A launch
// covers 3 NW shells (60 at 640 threads, 72 at 768); more shells take one
// launch per window (phase 1 reads all shells in each).  With EXT, e comes from summed subvolume partials E_p (e =
// E_p - C, the same double-float subtraction as k_kappa_finish) and the
// counts, those of one subvolume, enter phase 1 only through their maximum:
// the per-shell sums are then that subvolume's share, and they add over
// subvolumes.
// Block sizes (4 pixels per thread, 3 shells per warp): 640 threads (2560-
// pixel tiles, 60 shells per launch) for maps of up to 60 shells, 768 (3072-
// pixel tiles, 72 shells) above.  Measured at 60 shells, Nside 1024: 1024
// threads 1.34 ms, 896 1.34, 832 1.30, 768 1.08, 704 1.20, 640 1.04 (12
// shells unrolled in phase 1); the tiles in flight of the smaller blocks
// (152 x 2560 pixels x 60 shells x 4 B = 93 MB) stay in L2 for phase 2.
constexpr int kAdjThreadsSmall = 640;
constexpr int kAdjThreadsLarge = 768;
constexpr int kAdjSpw = 3;                // shells per warp in phase 2

template <bool USE_G, int NT, bool EXT>
__global__ void __launch_bounds__(NT, 1)
k_adj_main(const int32_t* __restrict__ counts, Coef cf, const float* __restrict__ g,
           double* __restrict__ rows_out, double* __restrict__ sumpart,
           unsigned long long* range_flag, int s0, float* __restrict__ kappa_out,
           double* __restrict__ ksum_out, const double* __restrict__ ext) {
  extern __shared__ __align__(16) uint8_t adj_sm[];
  constexpr int T = NT, NW = T / 32, TP = 4 * T;
  int* q_s = reinterpret_cast<int*>(adj_sm);                 // [6][TP] quantised e, e^2, g
  float* ef_s = reinterpret_cast<float*>(adj_sm);            // the same memory: e, e^2 as floats
  float* ps_s = reinterpret_cast<float*>(adj_sm + 24 * TP);   // [8][T] this thread's power sums
  AdjRow* rows = reinterpret_cast<AdjRow*>(adj_sm + 24 * TP + 32 * T);  // [nshell]
  __shared__ float ah_s[kMaxShells], al_s[kMaxShells];
  __shared__ float mred[3][NW];
  __shared__ int nred[NW];
  __shared__ double red[NW];
  const int S = cf.nshell, npix = cf.npix, ng = npix >> 2;
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  for (int i = threadIdx.x; i < S; i += T) { ah_s[i] = cf.ah[i]; al_s[i] = cf.al[i]; rows[i] = AdjRow{}; }
  // running maxima of |e|, e^2, |g| over this block's tiles, in shared
  // memory: thread 0 updates them after a barrier that every thread's read
  // of them for the tile has passed
  __shared__ float Ms[3];
  if (threadIdx.x == 0) Ms[0] = Ms[1] = Ms[2] = 0.f;
  auto scale = [](float M) { return M > 0.f ? min(120, 21 - ilog2f(M)) : 0; };
  for (int k = 0; k < 8; ++k) ps_s[k * T + threadIdx.x] = 0.f;
  __syncthreads();                         // ah_s, al_s, rows and Ms before any use
  constexpr int NQ = USE_G ? 6 : 4;
  long long acc[kAdjSpw][NQ + 1];
#pragma unroll
  for (int k = 0; k < kAdjSpw; ++k)
#pragma unroll
    for (int j = 0; j <= NQ; ++j) acc[k][j] = 0;
  auto flush = [&](int s1, int s2, int s3) {
#pragma unroll
    for (int k = 0; k < kAdjSpw; ++k) {
      const int b = s0 + w + NW * k;
      long long a[NQ + 1];
#pragma unroll
      for (int j = 0; j <= NQ; ++j) { a[j] = warp_sum_ll(acc[k][j]); acc[k][j] = 0; }
      if (ln == 0 && b < S) {
        AdjRow& row = rows[b];
        i128_add(row.s[0], a[0], kFrac1 - s1);
        i128_add(row.s[0], a[1], kFrac1 - s1 - 22);
        i128_add(row.s[1], a[2], kFrac2 - s2);
        i128_add(row.s[1], a[3], kFrac2 - s2 - 22);
        if (USE_G) {
          i128_add(row.s[2], a[4], kFrac3 - s3);
          i128_add(row.s[2], a[5], kFrac3 - s3 - 22);
        }
        row.n += a[NQ];
      }
    }
  };
  const int4* c4 = reinterpret_cast<const int4*>(counts);
  const f2 mc{-cf.ch, -cf.cl};
  const int ntile = (npix + TP - 1) / TP;
  double bound = 0.0;                      // bound on |any 64-bit sum|, uniform
  f2 ks{0.f, 0.f};                         // this thread's sum of the FP32 map (kappa_out)
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    // phase 1: e of 4 adjacent pixels per thread (the shells in order, as in
    // the forward pass), the power sums and the tile's maxima; e and e^2
    // wait in shared memory until the tile's scale is known
    const int gi = tile * T + threadIdx.x;   // group of 4 pixels
    const bool have = gi < ng;
    f2 a[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int nmx = 0;
    if (have) {
      // shells unrolled for loads in flight (fewer with g, whose registers
      // would spill more)
      constexpr int kU1 = USE_G ? 6 : 12;
#pragma unroll kU1
      for (int b = 0; b < S; ++b) {
        const int4 n = c4[(size_t)b * ng + gi];
        nmx = max(nmx, max(max(n.x, n.y), max(n.z, n.w)));
        if constexpr (!EXT) {
          const float h = ah_s[b], l = al_s[b];
          f2_mac(a[0], h, l, float(n.x));
          f2_mac(a[1], h, l, float(n.y));
          f2_mac(a[2], h, l, float(n.z));
          f2_mac(a[3], h, l, float(n.w));
        }
      }
      if constexpr (EXT) {
        const double2 d01 = reinterpret_cast<const double2*>(ext)[2 * gi];
        const double2 d23 = reinterpret_cast<const double2*>(ext)[2 * gi + 1];
        a[0] = d_to_f2(d01.x);
        a[1] = d_to_f2(d01.y);
        a[2] = d_to_f2(d23.x);
        a[3] = d_to_f2(d23.y);
      }
    }
    const float4 gv4 = (USE_G && have) ? reinterpret_cast<const float4*>(g)[gi]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
    const float gs[4] = {gv4.x, gv4.y, gv4.z, gv4.w};
    float t1 = 0.f, t2 = 0.f, t3 = 0.f;
    float kv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f2 e = f2_add(f2_norm(a[i].h, a[i].l), mc);
      kv[i] = __fadd_rn(e.h, e.l);             // the FP32 map, as the forward pass rounds it
      f2 e2 = f2_mul(e, e);
      if (!have) { e = f2{0.f, 0.f}; e2 = f2{0.f, 0.f}; }
      t1 = fmaxf(t1, fabsf(e.h));
      t2 = fmaxf(t2, fabsf(e2.h));
      t3 = fmaxf(t3, fabsf(gs[i]));
      const int px = 4 * threadIdx.x + i;
      ef_s[px] = e.h;
      ef_s[TP + px] = e.l;
      ef_s[2 * TP + px] = e2.h;
      ef_s[3 * TP + px] = e2.l;
    }
    if (kappa_out && have) {                   // (uniform) the map itself, with its sum
      reinterpret_cast<float4*>(kappa_out)[gi] = make_float4(kv[0], kv[1], kv[2], kv[3]);
      ks = f2_add(ks, f2_add(f2_two_sum(kv[0], kv[1]), f2_two_sum(kv[2], kv[3])));
    }
    if (have) {
      f2 p1{ps_s[threadIdx.x], ps_s[T + threadIdx.x]};
      f2 p2{ps_s[2 * T + threadIdx.x], ps_s[3 * T + threadIdx.x]};
      f2 p3{ps_s[4 * T + threadIdx.x], ps_s[5 * T + threadIdx.x]};
      f2 qg{ps_s[6 * T + threadIdx.x], ps_s[7 * T + threadIdx.x]};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int px = 4 * threadIdx.x + i;
        const f2 e{ef_s[px], ef_s[TP + px]};
        const f2 e2{ef_s[2 * TP + px], ef_s[3 * TP + px]};
        p1 = f2_add(p1, e);
        p2 = f2_add(p2, e2);
        p3 = f2_add(p3, f2_mul(e2, e));
        qg = f2_add(qg, f2{gs[i], 0.f});
      }
      ps_s[threadIdx.x] = p1.h; ps_s[T + threadIdx.x] = p1.l;
      ps_s[2 * T + threadIdx.x] = p2.h; ps_s[3 * T + threadIdx.x] = p2.l;
      ps_s[4 * T + threadIdx.x] = p3.h; ps_s[5 * T + threadIdx.x] = p3.l;
      ps_s[6 * T + threadIdx.x] = qg.h; ps_s[7 * T + threadIdx.x] = qg.l;
    }
    for (int o = 16; o > 0; o >>= 1) {
      nmx = max(nmx, __shfl_xor_sync(0xFFFFFFFFu, nmx, o));
      t1 = fmaxf(t1, __shfl_xor_sync(0xFFFFFFFFu, t1, o));
      t2 = fmaxf(t2, __shfl_xor_sync(0xFFFFFFFFu, t2, o));
      t3 = fmaxf(t3, __shfl_xor_sync(0xFFFFFFFFu, t3, o));
    }
    if (ln == 0) { nred[w] = nmx; mred[0][w] = t1; mred[1][w] = t2; mred[2][w] = t3; }
    __syncthreads();
    int NMX = 0;
    float T1 = 0.f, T2 = 0.f, T3 = 0.f;
    for (int i = 0; i < NW; ++i) {
      NMX = max(NMX, nred[i]);
      T1 = fmaxf(T1, mred[0][i]);
      T2 = fmaxf(T2, mred[1][i]);
      T3 = fmaxf(T3, mred[2][i]);
    }
    const float M1 = Ms[0], M2 = Ms[1], M3 = Ms[2];
    const bool grow = T1 > M1 || T2 > M2 || T3 > M3;   // (uniform) a coarser scale
    const double inc = double(TP / 32) * double(NMX) * 4194304.0;   // per lane, this tile
    if (grow || bound + inc > 2305843009213693952.0) {              // 2^61
      flush(scale(M1), scale(M2), scale(M3));                       // at the old scale
      bound = 0.0;
    }
    bound += inc;
    const float N1 = fmaxf(M1, T1), N2 = fmaxf(M2, T2), N3 = fmaxf(M3, T3);
    if (grow && threadIdx.x == 0 && (N1 >= 16384.0f || N3 >= 16384.0f || N2 >= 268435456.0f))
      atomicAdd(range_flag, 1ull);
    const int s1 = scale(N1), s2 = scale(N2), s3 = scale(N3);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int px = 4 * threadIdx.x + i;
      const f2 e{ef_s[px], ef_s[TP + px]};
      const f2 e2{ef_s[2 * TP + px], ef_s[3 * TP + px]};
      int h, l;
      quant2(e, s1, h, l);
      q_s[px] = h;
      q_s[TP + px] = l;
      quant2(e2, s2, h, l);
      q_s[2 * TP + px] = h;
      q_s[3 * TP + px] = l;
      if (USE_G) {
        quant2(f2{gs[i], 0.f}, s3, h, l);
        q_s[4 * TP + px] = h;
        q_s[5 * TP + px] = l;
      }
    }
    __syncthreads();                       // q_s complete; every thread has read Ms
    if (grow && threadIdx.x == 0) { Ms[0] = N1; Ms[1] = N2; Ms[2] = N3; }
    // phase 2: lane ln takes pixels ln, ln + 32, ... of the tile (L2 re-reads)
    const int base = tile * TP;
    const int valid = min(TP, npix - base);
#pragma unroll 16
    for (int pi = ln; pi < valid; pi += 32) {          // 48 count loads in flight per lane
      int qv[NQ];
#pragma unroll
      for (int j = 0; j < NQ; ++j) qv[j] = q_s[j * TP + pi];
#pragma unroll
      for (int k = 0; k < kAdjSpw; ++k) {
        const int b = s0 + w + NW * k;
        if (b < S) {
          const long long n = counts[(size_t)b * npix + base + pi];
#pragma unroll
          for (int j = 0; j < NQ; ++j) acc[k][j] += (long long)qv[j] * n;
          acc[k][NQ] += n;
        }
      }
    }
    __syncthreads();                       // q_s and nred are rewritten by the next tile
  }
  __syncthreads();
  flush(scale(Ms[0]), scale(Ms[1]), scale(Ms[2]));
  __syncthreads();
  double* dst = rows_out + (size_t)blockIdx.x * 4 * S;
  const int s_end = min(S, s0 + kAdjSpw * NW);   // the shells of this launch: [s0, s_end)
  for (int b = s0 + threadIdx.x; b < s_end; b += T) {
    dst[4 * b + 0] = i128_to_d(rows[b].s[0], kFrac1);
    dst[4 * b + 1] = i128_to_d(rows[b].s[1], kFrac2);
    dst[4 * b + 2] = USE_G ? i128_to_d(rows[b].s[2], kFrac3) : 0.0;
    dst[4 * b + 3] = (double)rows[b].n;
  }
  const f2 p1{ps_s[threadIdx.x], ps_s[T + threadIdx.x]}, p2{ps_s[2 * T + threadIdx.x], ps_s[3 * T + threadIdx.x]};
  const f2 p3{ps_s[4 * T + threadIdx.x], ps_s[5 * T + threadIdx.x]}, qg{ps_s[6 * T + threadIdx.x], ps_s[7 * T + threadIdx.x]};
  if (kappa_out) {                         // (uniform)
    const double vk = block_sum_d<T>(f2_to_d(ks), red);
    if (threadIdx.x == 0) ksum_out[blockIdx.x] = vk;
  }
  const double v1 = block_sum_d<T>(f2_to_d(p1), red);
  if (threadIdx.x == 0) sumpart[4 * blockIdx.x + 0] = v1;
  const double v2 = block_sum_d<T>(f2_to_d(p2), red);
  if (threadIdx.x == 0) sumpart[4 * blockIdx.x + 1] = v2;
  const double v3 = block_sum_d<T>(f2_to_d(p3), red);
  if (threadIdx.x == 0) sumpart[4 * blockIdx.x + 2] = v3;
  const double v4 = block_sum_d<T>(f2_to_d(qg), red);
  if (threadIdx.x == 0) sumpart[4 * blockIdx.x + 3] = v4;
}

// Per-block sums of an FP32 map (double-float per thread), the first pass of
// the moments of an arbitrary map (ufc_map_stats).  Needs a 16-byte aligned
// map of a multiple of 4 values.
__global__ void __launch_bounds__(kKV)
k_map_sum(const float* __restrict__ map, int npix, double* __restrict__ ksum_part) {
  __shared__ double red[kKV / 32];
  const int ng = npix >> 2;
  f2 ks{0.f, 0.f};
  for (int g = blockIdx.x * kKV + threadIdx.x; g < ng; g += gridDim.x * kKV) {
    const float4 v = reinterpret_cast<const float4*>(map)[g];
    ks = f2_add(ks, f2_add(f2_two_sum(v.x, v.y), f2_two_sum(v.z, v.w)));
  }
  const double t = block_sum_d<kKV>(f2_to_d(ks), red);
  if (threadIdx.x == 0) ksum_part[blockIdx.x] = t;
}

// ------------------------------------------------ moments + PDF pass -----
// Second pass over the FP32 map (L2-resident at these sizes): central
// power sums about the exact FP64 mean in double-float, and the PDF.
// PDF bin = floor((kappa - lo) * scale) in FP64; an FP32 estimate decides
// all but the values within a proven band of a bin edge.
constexpr int kMT = 256;
constexpr int kMaxBins = 4096;

struct PdfParam {
  double lo, hi, scale;     // scale = nbins / (hi - lo)
  float lo_f, scale_f, band_rel;
  float lo_dn, lo_up, hi_dn, hi_up;   // FP32 brackets of lo and hi
  int32_t nbins;
};

// Sum of v[0], v[stride], ..., v[(n - 1) stride] by one warp in a fixed
// order: lane l adds elements l, l + 32, ... in turn, then a butterfly; every
// lane ends with the same value (each pairwise sum is formed by both lanes).
__device__ __forceinline__ double warp_sum_fixed(const double* v, int n, int stride) {
  double s = 0.0;
  for (int i = threadIdx.x & 31; i < n; i += 32) s += v[(size_t)i * stride];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  return s;
}

// PDF slot of one FP32 value: floor((k - lo) * scale) in FP64, decided in FP32
// unless k lies within a proven band of a bin edge; under/overflow and NaN.
__device__ __forceinline__ int pdf_slot(float k, const PdfParam& pp) {
  // k < lo and k >= hi decided in FP32 unless k lies between the FP32
  // neighbours of lo (resp. hi)
  const bool under = k < pp.lo_dn || (k < pp.lo_up && (double)k < pp.lo);
  const bool over = k >= pp.hi_up || (k >= pp.hi_dn && (double)k >= pp.hi);
  if (isnan(k)) return pp.nbins + 2;
  if (under) return pp.nbins;
  if (over) return pp.nbins + 1;
  const float x = (k - pp.lo_f) * pp.scale_f;   // in [-1, nbins + 1] up to rounding
  float xr;
  int b = round_fast(x, xr);
  if (xr > x) { b -= 1; xr -= 1.0f; }          // floor
  const float rem = x - xr;
  const float band = pp.band_rel * (fabsf(x) + 1.0f);
  if (!(rem >= band && rem < 1.0f - band))
    b = (int)floor(__dmul_rn(__dsub_rn((double)k, pp.lo), pp.scale));
  return b >= pp.nbins ? pp.nbins - 1 : (b < 0 ? 0 : b);
}

// One block's share of the moment pass: block vb of a grid of nb blocks of
// kMT threads (every thread calls it).  Central power sums about `mean` into
// out[0..2] (valid in thread 0); PDF counts into the shared histogram.
__device__ __forceinline__ void moments_block(const float* __restrict__ kappa, int npix,
                                              double mean, const PdfParam& pp, int vb, int nb,
                                              unsigned int* hist, double* red, double* out) {
  const float mh = (float)mean;
  const float ml = (float)(mean - (double)mh);
  f2 a2{0.f, 0.f}, a3{0.f, 0.f}, a4{0.f, 0.f};
  for (int p = vb * kMT + threadIdx.x; p < npix; p += nb * kMT) {
    const float k = kappa[p];
    f2 d = f2_add(f2_two_sum(k, -mh), f2{-ml, 0.f});
    f2 d2 = f2_mul(d, d);
    a2 = f2_add(a2, d2);
    a3 = f2_add(a3, f2_mul(d2, d));
    a4 = f2_add(a4, f2_mul(d2, d2));
    atomicAdd(hist + pdf_slot(k, pp), 1u);
  }
  out[0] = block_sum_d<kMT>(f2_to_d(a2), red);
  out[1] = block_sum_d<kMT>(f2_to_d(a3), red);
  out[2] = block_sum_d<kMT>(f2_to_d(a4), red);
}

__global__ void __launch_bounds__(kMT)
k_moments(const float* __restrict__ kappa, int npix, const double* __restrict__ ksum_part,
          int nksum, PdfParam pp, double* __restrict__ part /*[grid][3]*/,
          unsigned long long* __restrict__ pdf /*[nbins+3]*/) {
  extern __shared__ unsigned int hist[];   // [nbins + 3]
  __shared__ double red[kMT / 32];
  __shared__ double mean_s;
  for (int i = threadIdx.x; i < pp.nbins + 3; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x < 32) {
    const double s = warp_sum_fixed(ksum_part, nksum, 1);   // fixed order
    if (threadIdx.x == 0) mean_s = s / double(npix);
  }
  __syncthreads();
  double o[3];
  moments_block(kappa, npix, mean_s, pp, blockIdx.x, gridDim.x, hist, red, o);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = o[0];
    part[3 * blockIdx.x + 1] = o[1];
    part[3 * blockIdx.x + 2] = o[2];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < pp.nbins + 3; i += blockDim.x)
    if (hist[i]) atomicAdd(pdf + i, (unsigned long long)hist[i]);
}

// moments[10] from the partial sums (one warp, fixed orders; every lane of
// warp 0 calls it, lane 0 writes).
__device__ __forceinline__ void moments_final_warp(const double* ksum_part, int nksum,
                                                   const double* part, int npart, int npix,
                                                   double* m) {
  // the mean as k_moments forms it
  const double s = warp_sum_fixed(ksum_part, nksum, 1);
  const double s2 = warp_sum_fixed(part, npart, 3);
  const double s3 = warp_sum_fixed(part + 1, npart, 3);
  const double s4 = warp_sum_fixed(part + 2, npart, 3);
  if (threadIdx.x != 0) return;
  const double N = double(npix);
  const double mu2 = s2 / N, mu3 = s3 / N, mu4 = s4 / N;
  m[0] = s / N;
  m[1] = mu2;
  m[2] = mu3;
  m[3] = mu4;
  m[4] = mu3 / (mu2 * sqrt(mu2));
  m[5] = mu4 / (mu2 * mu2) - 3.0;
  m[6] = (N - 1.0) * mu2 / N;
  // Eq. 13 with every product and difference rounded on its own (explicit
  // intrinsics: no contraction can differ between the copies of this code)
  const double N3 = __dmul_rn(__dmul_rn(N, N), N);
  const double c1 = __ddiv_rn(__dmul_rn(N - 1.0, N - 1.0), N3);
  const double c2 = __ddiv_rn(__dmul_rn(N - 1.0, N - 3.0), N3);
  m[7] = __dsub_rn(__dmul_rn(c1, mu4), __dmul_rn(__dmul_rn(c2, mu2), mu2));
  m[8] = mu2 / m[7];
  m[9] = N;
}

__global__ void k_moments_final(const double* __restrict__ ksum_part, int nksum,
                                const double* __restrict__ part, int npart, int npix,
                                double* __restrict__ m) {
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  moments_final_warp(ksum_part, nksum, part, npart, npix, m);
}

// Statistics vector of one map for the covariance (Eq. 10): the first six
// moments (mean, mu2, mu3, mu4, skew, kurtosis) then the PDF bins divided by
// the pixel count.
__global__ void k_stats_vector(const double* __restrict__ m, const unsigned long long* __restrict__ pdf,
                               int nbins, double* __restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 6 + nbins; i += gridDim.x * blockDim.x)
    v[i] = i < 6 ? m[i] : double(pdf[i - 6]) / m[9];
}

// ---------------------------------------------------------- Welford -----
// Welford update of st by the nvec vectors v [nvec][d] in order (every thread
// of the block calls it; sh holds 2 rc d doubles).  Runs of rc vectors: the
// deltas of each vector against the running mean (dold = x - mean before,
// dnew = x - mean after) are formed in order into shared memory, the mean
// updated as they are; then every element of M2 takes the run's products
// as one chain of fused multiply-adds in a register, one global read and
// write per run instead of per vector.  The chain per element is the same as
// one vector at a time, so the result does not depend on rc or on the block
// size.  The count is read once and written once.
__device__ __forceinline__ void welford_update_block(const double* v, int nvec, int d, double* st,
                                                     double* sh, int rc) {
  double* mean = st + 1;
  double* M2 = st + 1 + d;
  const double n0 = st[0];
  __syncthreads();
  for (int r0 = 0; r0 < nvec; r0 += rc) {
    const int nr = min(rc, nvec - r0);
    // the run's deltas, in vector order (thread i owns mean[i] throughout)
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
      double m = mean[i];
      for (int q = 0; q < nr; ++q) {
        const double x = v[(size_t)(r0 + q) * d + i];
        const double n = n0 + double(r0 + q + 1);
        const double delta = x - m;
        m = m + delta / n;
        sh[(size_t)q * d + i] = delta;                 // dold
        sh[(size_t)(rc + q) * d + i] = x - m;          // dnew
      }
      mean[i] = m;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < d * d; k += blockDim.x) {
      const int i = k / d, j = k - i * d;
      double acc = M2[k];
      for (int q = 0; q < nr; ++q)
        acc = __fma_rn(sh[(size_t)q * d + i], sh[(size_t)(rc + q) * d + j], acc);
      M2[k] = acc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) st[0] = n0 + double(nvec);
}

// Vectors per run of the Welford update for d-dimensional states: the run's
// deltas (2 rc d doubles) within 48 KB of shared memory, at most 16.
__host__ __device__ inline int welford_run(int d) {
  const int rc = 49152 / (16 * d);
  return rc < 1 ? 1 : (rc > 16 ? 16 : rc);
}

__global__ void __launch_bounds__(1024)
k_welford_update(const double* __restrict__ v, int nvec, int d, double* __restrict__ st) {
  extern __shared__ double sh[];   // the run's deltas: dold[rc][d], dnew[rc][d]
  welford_update_block(v, nvec, d, st, sh, welford_run(d));
}

__global__ void __launch_bounds__(1024)
k_welford_merge(double* __restrict__ a, const double* __restrict__ b, int d) {
  const double na = a[0], nb = b[0], n = na + nb;
  if (nb == 0.0) return;
  double* ma = a + 1;
  const double* mb = b + 1;
  double* Ma = a + 1 + d;
  const double* Mb = b + 1 + d;
  const double f = (n > 0.0) ? na * nb / n : 0.0;
  for (int k = threadIdx.x; k < d * d; k += blockDim.x) {
    const int i = k / d, j = k - i * d;
    Ma[k] += Mb[k] + (mb[i] - ma[i]) * (mb[j] - ma[j]) * f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) ma[i] += (mb[i] - ma[i]) * nb / n;
  __syncthreads();
  if (threadIdx.x == 0) a[0] = n;
}

__global__ void __launch_bounds__(1024)
k_welford_final(const double* __restrict__ st, int d, int ddof, double* __restrict__ mean,
                double* __restrict__ cov, double* __restrict__ corr) {
  const double n = st[0];
  const double den = n - double(ddof);
  for (int i = threadIdx.x; i < d; i += blockDim.x) mean[i] = st[1 + i];
  for (int k = threadIdx.x; k < d * d; k += blockDim.x) cov[k] = st[1 + d + k] / den;
  __syncthreads();
  for (int k = threadIdx.x; k < d * d; k += blockDim.x) {
    const int i = k / d, j = k - i * d;
    const double q = sqrt((st[1 + d + i * d + i] / den) * (st[1 + d + j * d + j] / den));
    corr[k] = q > 0.0 ? (st[1 + d + k] / den) / q : 0.0;
  }
}

// ------------------------------------------------ persistent batch kernel --
// All realisations of a batched call (Sec. 3.2: statistics over many
// realisations) in one launch.  A device work queue hands out tasks of
// `chunk` particles of one (realisation, box); a block bins its task's
// particles with the three-stage key (FP32, double-float and FP64 stages
// inline: the same keys as the binning call) and adds them to the
// realisation's count map with global atomics.  The block that finishes the
// last task of a realisation then computes its kappa map, moments, PDF and
// statistics vector by running, one after the other, every block of the
// serial kappa and moment passes (kappa_vec_block and moments_block with the
// serial grids), so that the results equal the one-at-a-time calls bit for
// bit.  The block that finishes the last realisation runs the Welford
// update over all of them in realisation order.  No block ever waits for
// another one: completion is detected with atomic counters and fences.
struct BatchItem {          // one (realisation, box) of a batched call
  const float* xyz;
  int64_t n;
  int64_t task0;            // first task of this item (ascending over the items)
  int32_t real;
  int32_t shell_lo, shell_hi;
  float shf[3], shlo[3];    // the box's shift split as in BoxGeom (no periodic images)
  double sh64[3];
};
struct BatchArgs {
  const BatchItem* items;
  int32_t nitems, chunk;
  int64_t ntasks;
  const Coef* coef;         // [nreal]
  const int32_t* ntask_r;   // [nreal] tasks of each realisation
  int32_t nreal, S, N, npix;
  int32_t* counts;          // [nreal][S][npix], zero at the launch
  float* kappa;             // [nreal][npix]
  double* ksum;             // [nreal][gk]
  double* mpart;            // [nreal][3 gm]
  int32_t gk, gm;           // grids of the serial kappa and moment passes
  double* moments;          // [nreal][10]
  int64_t* pdf;             // [nreal][nbins + 3]
  double* stats;            // [nreal][d]
  double* state;            // Welford state (1 + d + d^2)
  int32_t nbins, d;
  unsigned long long* queue;   // [0] next task, [1] realisations finished (zero at launch)
  unsigned int* done;          // [nreal] tasks finished (zero at launch)
};
constexpr int kBT = 256;
static_assert(kBT == kKV && kBT == kMT, "the persistent blocks reproduce the serial blocks");

// Key of one particle: FP32 stage, then the double-float and FP64 stages for
// what it leaves undecided (shell_fast: binary search over the FP32 bands).
__device__ __forceinline__ int32_t batch_key(float x, float y, float zc, const BatchItem& it,
                                             const float* lo2, const float* hi2,
                                             const float* chih, const float* chil,
                                             const float2* atab,
                                             const ShellTable& st, const Bands& bd, int32_t N,
                                             int32_t npix) {
  const int lo = it.shell_lo, hi = it.shell_hi;
  const float dx = (x + it.shf[0]) + it.shlo[0];
  const float dy = (y + it.shf[1]) + it.shlo[1];
  const float dz = (zc + it.shf[2]) + it.shlo[2];
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  int32_t key = kKeyUndecided;
  if (r2 >= bd.r2_min && r2 <= 3.0e38f) {
    const int32_t b = shell_fast(lo2, hi2, lo, hi, r2);
    if (b == -1) {
      key = kKeyOutside;
    } else if (b >= 0) {
      const int32_t pix = pixel_fast(N, bd, dx, dy, dz, r2);
      if (pix != kKeyUndecided) key = b * npix + pix;
    }
  }
  if (key == kKeyUndecided)
    key = key_refine(chih, chil, atab, lo, hi, N, npix, x, y, zc, it.shf[0], it.shf[1], it.shf[2], it.shlo[0],
                     it.shlo[1], it.shlo[2]);
  if (key == kKeyUndecided)
    key = key_exact(st, lo, hi, N, npix, x, y, zc, it.sh64[0], it.sh64[1], it.sh64[2]);
  return key;
}

__global__ void __launch_bounds__(kBT)
k_batch_persistent(BatchArgs ba, ShellTable st, Bands bd, PdfParam pp) {
  extern __shared__ __align__(16) uint8_t bsm[];   // PDF histogram, then Welford scratch
  __shared__ float lo2_s[kMaxShells + 2], hi2_s[kMaxShells + 2];
  __shared__ float chih_s[kMaxShells + 1], chil_s[kMaxShells + 1];
  __shared__ float2 atab_s[kAtanTab];
  __shared__ float ah_s[kMaxShells], al_s[kMaxShells];
  __shared__ double red[kBT / 32];
  __shared__ long long task_s;
  __shared__ int flag_s;
  __shared__ double mean_s;
  for (int i = threadIdx.x; i <= st.nshell; i += kBT) {
    lo2_s[i] = st.lo2[i];
    hi2_s[i] = st.hi2[i];
    chih_s[i] = st.chih[i];
    chil_s[i] = st.chil[i];
  }
  fill_atan_table(atab_s);                 // (the task loop's first barrier follows)
  const int S = ba.S, npix = ba.npix, ng = npix >> 2;
  for (;;) {
    if (threadIdx.x == 0) task_s = (long long)atomicAdd(&ba.queue[0], 1ull);
    __syncthreads();
    const long long t = task_s;
    if (t >= ba.ntasks) break;
    // the task's item: the last one whose first task is <= t
    int a = 0, b = ba.nitems;
    while (b - a > 1) {
      const int m = (a + b) >> 1;
      if (ba.items[m].task0 <= t) a = m; else b = m;
    }
    const BatchItem it = ba.items[a];
    const int r = it.real;
    const int64_t p0 = (t - it.task0) * ba.chunk;
    const int64_t cnt = min((int64_t)ba.chunk, it.n - p0);
    int32_t* cmap = ba.counts + (size_t)r * S * npix;
    for (int64_t i = threadIdx.x; i < cnt; i += kBT) {
      const float* q = it.xyz + 3 * (p0 + i);
      const int32_t key = batch_key(__ldg(q), __ldg(q + 1), __ldg(q + 2), it, lo2_s, hi2_s,
                                    chih_s, chil_s, atab_s, st, bd, ba.N, npix);
      if (key >= 0 && UFC_IDX_OK(key, (int64_t)S * npix, 8)) atomicAdd(cmap + key, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();                       // this block's keys before its count of the task
      flag_s = atomicAdd(&ba.done[r], 1u) == (unsigned)(ba.ntask_r[r] - 1);
    }
    __syncthreads();
    if (!flag_s) continue;
    // ---- the last task of realisation r: its map, moments, PDF, statistics
    __threadfence();                         // every block's keys of r are visible
    const Coef& cf = ba.coef[r];
    for (int i = threadIdx.x; i < S; i += kBT) { ah_s[i] = cf.ah[i]; al_s[i] = cf.al[i]; }
    __syncthreads();
    const f2 mc{-cf.ch, -cf.cl};
    float* kap = ba.kappa + (size_t)r * npix;
    double* ks = ba.ksum + (size_t)r * ba.gk;
    for (int vb = 0; vb < ba.gk; ++vb) {
      if (vb * kKV < ng) {                   // uniform; the serial blocks past the map add 0.0
        const double v = kappa_vec_block(cmap, ah_s, al_s, S, npix, mc, kap, vb, ba.gk, red);
        if (threadIdx.x == 0) ks[vb] = v;
      } else if (threadIdx.x == 0) {
        ks[vb] = 0.0;
      }
    }
    unsigned int* hist = reinterpret_cast<unsigned int*>(bsm);
    for (int i = threadIdx.x; i < ba.nbins + 3; i += kBT) hist[i] = 0u;
    __syncthreads();
    if (threadIdx.x < 32) {
      const double sum = warp_sum_fixed(ks, ba.gk, 1);      // fixed order, as k_moments
      if (threadIdx.x == 0) mean_s = sum / double(npix);
    }
    __syncthreads();
    double* mp = ba.mpart + (size_t)r * 3 * ba.gm;
    for (int vb = 0; vb < ba.gm; ++vb) {
      if (vb * kMT < npix) {
        double o[3];
        moments_block(kap, npix, mean_s, pp, vb, ba.gm, hist, red, o);
        if (threadIdx.x == 0) { mp[3 * vb] = o[0]; mp[3 * vb + 1] = o[1]; mp[3 * vb + 2] = o[2]; }
      } else if (threadIdx.x == 0) {
        mp[3 * vb] = 0.0; mp[3 * vb + 1] = 0.0; mp[3 * vb + 2] = 0.0;
      }
    }
    __syncthreads();
    double* mo = ba.moments + 10 * (size_t)r;
    int64_t* pd = ba.pdf + (size_t)(ba.nbins + 3) * r;
    if (threadIdx.x < 32) moments_final_warp(ks, ba.gk, mp, ba.gm, npix, mo);
    for (int i = threadIdx.x; i < ba.nbins + 3; i += kBT) pd[i] = (int64_t)hist[i];
    __syncthreads();
    double* v = ba.stats + (size_t)ba.d * r;
    for (int i = threadIdx.x; i < ba.d; i += kBT) v[i] = i < 6 ? mo[i] : double(pd[i - 6]) / mo[9];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();                       // r's results before its count
      flag_s = atomicAdd(&ba.queue[1], 1ull) == (unsigned long long)(ba.nreal - 1);
    }
    __syncthreads();
    if (flag_s) {                            // the last realisation: the covariance update
      __threadfence();
      welford_update_block(ba.stats, ba.nreal, ba.d, ba.state, reinterpret_cast<double*>(bsm),
                           welford_run(ba.d));
    }
    __syncthreads();
  }
}

// ============================================================== host =====

// Index-check record of this translation unit (checked builds), read and
// cleared on the context stream.
cudaError_t take_checks_stats(CheckRec* out, cudaStream_t s) { return take_check_rec(out, s); }

static void make_coef(const double* A, double C, int S, int npix, Coef& cf) {
  std::memset(&cf, 0, sizeof cf);
  for (int b = 0; b < S; ++b) {
    cf.ah[b] = (float)A[b];
    cf.al[b] = (float)(A[b] - (double)cf.ah[b]);
  }
  cf.ch = (float)C;
  cf.cl = (float)(C - (double)cf.ch);
  cf.nshell = S;
  cf.npix = npix;
}

static ufc_status check_kappa_args(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                   const double* A, double C) {
  if (!counts) return set_err(c, UFC_ERR_ARG, "counts_dev is NULL");
  if (S < 1 || S > kMaxShells) return set_err(c, UFC_ERR_ARG, "nshell must be in [1,%d]", kMaxShells);
  if (nside < 1 || nside > UFC_MAX_NSIDE || (nside & (nside - 1)))
    return set_err(c, UFC_ERR_ARG, "nside must be a power of two in [1,%d]", UFC_MAX_NSIDE);
  if ((int64_t)S * 12 * nside * nside >= (1ll << 31))
    return set_err(c, UFC_ERR_ARG, "nshell * 12 nside^2 must be < 2^31");
  if (!A) return set_err(c, UFC_ERR_ARG, "A is NULL");
  for (int b = 0; b < S; ++b)
    if (!std::isfinite(A[b])) return set_err(c, UFC_ERR_ARG, "A[%d] is not finite", b);
  if (!std::isfinite(C)) return set_err(c, UFC_ERR_ARG, "C is not finite");
  return UFC_OK;
}


// Forward kappa pass shared by ufc_kappa_stats and its allocation-free
// variant (identical results): grid blocks, one partial sum each in ksum.
static int kappa_fwd_grid(ufc_ctx* c) { return 8 * c->num_sms; }
static ufc_status launch_kappa_fwd(ufc_ctx* c, const int32_t* counts, const Coef& cf,
                                   float* kappa, double* ksum, int grid) {
  if ((reinterpret_cast<uintptr_t>(kappa) & 15) == 0) {
    k_kappa_vec<<<grid, kKV, 0, c->stream>>>(counts, cf, kappa, ksum);
  } else {
    k_kappa_plain<<<grid, kKT, 0, c->stream>>>(counts, cf, kappa, ksum);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}


// Moments and PDF of an FP32 map whose per-block sums (grid of them) are in
// ksum: the second pass over the map and the final reduction.
static PdfParam make_pdf_param(double lo, double hi, int nbins) {
  PdfParam pp;
  pp.lo = lo;
  pp.hi = hi;
  pp.scale = (double)nbins / (hi - lo);
  pp.lo_f = (float)lo;
  pp.scale_f = (float)pp.scale;
  pp.nbins = nbins;
  // |x_f - x_64| <= 3u |x| + u |lo| s + 2^-52 |x| (u = 2^-24); when
  // |lo| s < 16 that is below 68u (|x| + 1) < 2^-16 (|x| + 1), the band
  // used; other ranges send every value through the FP64 expression.
  pp.band_rel = std::fabs(lo) * pp.scale < 16.0 ? std::ldexp(1.0f, -16) : 2.0f;
  auto fdn = [](double v) { float f = (float)v; return (double)f > v ? nextafterf(f, -INFINITY) : f; };
  auto fup = [](double v) { float f = (float)v; return (double)f < v ? nextafterf(f, INFINITY) : f; };
  pp.lo_dn = fdn(lo);
  pp.lo_up = fup(lo);
  pp.hi_dn = fdn(hi);
  pp.hi_up = fup(hi);
  return pp;
}

static ufc_status launch_moments(ufc_ctx* c, const float* kmap, int npix, const double* ksum,
                                 int grid, double lo, double hi, int nbins, double* mpart,
                                 int mgrid, double* moments, int64_t* pdf, bool timed) {
  const PdfParam pp = make_pdf_param(lo, hi, nbins);
  UFC_CUDA(c, cudaMemsetAsync(pdf, 0, (size_t)(nbins + 3) * 8, c->stream));
  const int smem = (nbins + 3) * 4;
  {
    ProfScope ps_(timed ? c : nullptr, "k_moments");
    k_moments<<<mgrid, kMT, smem, c->stream>>>(kmap, npix, ksum, grid, pp, mpart,
                                               (unsigned long long*)pdf);
  }
  {
    ProfScope ps_(timed ? c : nullptr, "k_moments_final");
    k_moments_final<<<1, 32, 0, c->stream>>>(ksum, grid, mpart, mgrid, npix, moments);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

// Moments and PDF of any FP32 RING map (smoothed maps of Sec. 3.3).
ufc_status run_map_stats(ufc_ctx* c, const float* map, int nside, double lo, double hi,
                         int nbins, double* moments, int64_t* pdf) {
  if (!map || !moments || !pdf) return set_err(c, UFC_ERR_ARG, "map, moments and pdf are required");
  if (nside < 1 || nside > UFC_MAX_NSIDE || (nside & (nside - 1)))
    return set_err(c, UFC_ERR_ARG, "nside must be a power of two in [1,%d]", UFC_MAX_NSIDE);
  if (nbins < 1 || nbins > kMaxBins) return set_err(c, UFC_ERR_ARG, "nbins must be in [1,%d]", kMaxBins);
  if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
    return set_err(c, UFC_ERR_ARG, "PDF range needs finite lo < hi");
  if (reinterpret_cast<uintptr_t>(map) & 15) return set_err(c, UFC_ERR_ARG, "map_dev must be 16-byte aligned");
  const int npix = 12 * nside * nside;
  const int grid = kappa_fwd_grid(c), mgrid = 2 * c->num_sms;
  double* ksum = (double*)ws_get(c, kSlotPartials, (size_t)(grid + 3 * mgrid) * 8);
  if (!ksum) return UFC_ERR_ALLOC;
  {
    ProfScope ps_(c, "k_map_sum");
    k_map_sum<<<grid, kKV, 0, c->stream>>>(map, npix, ksum);
  }
  UFC_CUDA(c, cudaGetLastError());
  return launch_moments(c, map, npix, ksum, grid, lo, hi, nbins, ksum + grid, mgrid, moments, pdf,
                        true);
}

ufc_status run_kappa_stats(ufc_ctx* c, const int32_t* counts, int S, int nside,
                           const double* A, double C, double lo, double hi, int nbins,
                           float* kappa, double* moments, int64_t* pdf) {
  ufc_status s = check_kappa_args(c, counts, S, nside, A, C);
  if (s) return s;
  const int npix = 12 * nside * nside;
  const bool want_stats = moments || pdf;
  if (want_stats) {
    if (nbins < 1 || nbins > kMaxBins)
      return set_err(c, UFC_ERR_ARG, "nbins must be in [1,%d]", kMaxBins);
    if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
      return set_err(c, UFC_ERR_ARG, "PDF range needs finite lo < hi");
    if (!moments || !pdf)
      return set_err(c, UFC_ERR_ARG, "moments_dev and pdf_dev go together");
  }
  Coef cf;
  make_coef(A, C, S, npix, cf);
  if (reinterpret_cast<uintptr_t>(counts) & 15)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 16-byte aligned");
  const int grid = kappa_fwd_grid(c);
  const int mgrid = 2 * c->num_sms;
  double* ksum = (double*)ws_get(c, kSlotPartials, (size_t)(grid + 3 * mgrid) * 8);
  if (!ksum) return UFC_ERR_ALLOC;
  double* mpart = ksum + grid;
  float* kmap = kappa;
  if (!kmap && want_stats) {
    kmap = (float*)ws_get(c, kSlotMisc, (size_t)npix * 4);
    if (!kmap) return UFC_ERR_ALLOC;
  }
  if (!kmap) return UFC_OK;   // nothing requested
  {
    ProfScope ps_(c, "k_kappa");
    s = launch_kappa_fwd(c, counts, cf, kmap, ksum, grid);
    if (s) return s;
  }
  if (!want_stats) return UFC_OK;
  return launch_moments(c, kmap, npix, ksum, grid, lo, hi, nbins, mpart, mgrid, moments, pdf,
                        true);
}

// The adjoint's device pass and its reduction to the sums
// out[4 b + k] (b < S: S1_b = sum_p e_p n_bp, S2_b = sum_p e_p^2 n_bp,
// T_b = sum_p g_p n_bp, N_b = sum_p n_bp) and out[4 S + k] (P1, P2, P3 =
// sum_p e_p^k, Q = sum_p g_p).  e is built from the counts with A (ext NULL)
// or taken from summed subvolume partials ext (e = ext - C).  With kappa
// (non-NULL) the same launch writes the FP32 map and its block sums and the
// moment pass gives moments and PDF.  Synchronises.
static ufc_status adjoint_sums(ufc_ctx* c, const int32_t* counts, int S, int nside,
                               const Coef& cf, const double* ext, const float* g, float* kappa,
                               double lo, double hi, int nbins, double* moments, int64_t* pdf,
                               double* out) {
  if (kappa) {
    if (!moments || !pdf) return set_err(c, UFC_ERR_ARG, "moments_dev and pdf_dev are required");
    if (reinterpret_cast<uintptr_t>(kappa) & 15)
      return set_err(c, UFC_ERR_ARG, "kappa_dev must be 16-byte aligned");
    if (nbins < 1 || nbins > kMaxBins)
      return set_err(c, UFC_ERR_ARG, "nbins must be in [1,%d]", kMaxBins);
    if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
      return set_err(c, UFC_ERR_ARG, "PDF range needs finite lo < hi");
  }
  if (reinterpret_cast<uintptr_t>(counts) & 15)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 16-byte aligned");
  if (g && (reinterpret_cast<uintptr_t>(g) & 15))
    return set_err(c, UFC_ERR_ARG, "g_dev must be 16-byte aligned");
  if (ext && (reinterpret_cast<uintptr_t>(ext) & 15))
    return set_err(c, UFC_ERR_ARG, "partial_dev must be 16-byte aligned");
  const int npix = 12 * nside * nside;
  const int grid2 = c->num_sms;                            // one block per SM
  const size_t nrow = (size_t)grid2 * 4 * S, nsum = (size_t)grid2 * 4;
  const int mgrid = 2 * c->num_sms;
  const size_t nmap = kappa ? (size_t)grid2 + 3 * (size_t)mgrid : 0;   // map sums, moment partials
  double* part = (double*)ws_get(c, kSlotPartials, (nrow + nsum + nmap) * 8);
  if (!part) return UFC_ERR_ALLOC;
  double* rows = part;
  double* sums = part + nrow;
  double* ksum = sums + nsum;
  double* mpart = ksum + grid2;
  BinCounters* bc = reinterpret_cast<BinCounters*>(c->counters);
  UFC_CUDA(c, cudaMemsetAsync(&bc->range, 0, sizeof(unsigned long long), c->stream));
  // q_s, the threads' power sums, rows; one launch per window of shells
  // (a launch's warps own 3 shells each); every launch recomputes e from all
  // shells and writes the same power sums
  const bool small = S <= kAdjSpw * (kAdjThreadsSmall / 32);
  const int nt = small ? kAdjThreadsSmall : kAdjThreadsLarge;
  const int win = kAdjSpw * (nt / 32);
  const size_t smem2 = (size_t)24 * 4 * nt + (size_t)32 * nt + (size_t)S * sizeof(AdjRow);
  {
    ProfScope ps_(c, "k_adj_main");
#define UFC_ADJ(G, NT_, X)                                                                        \
  do {                                                                                            \
    UFC_CUDA(c, cudaFuncSetAttribute(k_adj_main<G, NT_, X>,                                       \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));   \
    for (int s0 = 0; s0 < S; s0 += win)                                                           \
      k_adj_main<G, NT_, X><<<grid2, NT_, smem2, c->stream>>>(                                    \
          counts, cf, g, rows, sums, &bc->range, s0, s0 == 0 ? kappa : nullptr, ksum, ext);       \
  } while (0)
#define UFC_ADJ_X(G, NT_)                                                                         \
  do {                                                                                            \
    if (ext) UFC_ADJ(G, NT_, true);                                                               \
    else UFC_ADJ(G, NT_, false);                                                                  \
  } while (0)
    if (g && small) UFC_ADJ_X(true, kAdjThreadsSmall);
    else if (g) UFC_ADJ_X(true, kAdjThreadsLarge);
    else if (small) UFC_ADJ_X(false, kAdjThreadsSmall);
    else UFC_ADJ_X(false, kAdjThreadsLarge);
#undef UFC_ADJ_X
#undef UFC_ADJ
  }
  UFC_CUDA(c, cudaGetLastError());
  if (kappa) {                             // moments and PDF of the map just written
    ufc_status s = launch_moments(c, kappa, npix, ksum, grid2, lo, hi, nbins, mpart, mgrid,
                                  moments, pdf, true);
    if (s) return s;
  }
  std::vector<double> hp(nrow + nsum);
  unsigned long long range_hits = 0;
  UFC_CUDA(c, cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  UFC_CUDA(c, cudaMemcpyAsync(&range_hits, &bc->range, 8, cudaMemcpyDeviceToHost, c->stream));
  UFC_CUDA(c, cudaStreamSynchronize(c->stream));
  if (range_hits)
    return set_err(c, UFC_ERR_UNSUPPORTED,
                   "adjoint needs |kappa_p| < 2^14 and |g_p| < 2^14 (fixed-point range)");
  for (int k = 0; k < 4 * S + 4; ++k) out[k] = 0.0;
  for (int i = 0; i < grid2; ++i) {        // blocks in order: a fixed summation order
    const double* r = hp.data() + (size_t)i * 4 * S;
    for (int k = 0; k < 4 * S; ++k) out[k] += r[k];
  }
  for (int i = 0; i < grid2; ++i) {
    const double* r = hp.data() + nrow + 4 * (size_t)i;
    for (int k = 0; k < 4; ++k) out[4 * S + k] += r[k];
  }
  return UFC_OK;
}

// dL/dtheta from the adjoint sums (layout of adjoint_sums), host FP64.
void grad_from_sums(const double* sm, int S, int npix, double w_var, double w_skew,
                    const double* dA, const double* dC, double* grad, double* G, double* H) {
  // central moments of the unrounded map from the raw sums about 0
  const double N = npix;
  const double P1 = sm[4 * S], P2 = sm[4 * S + 1], P3 = sm[4 * S + 2], Q = sm[4 * S + 3];
  const double m1 = P1 / N, r2 = P2 / N, r3 = P3 / N;
  const double mu2 = r2 - m1 * m1;
  const double mu3 = r3 - 3.0 * m1 * r2 + 2.0 * m1 * m1 * m1;
  // G_b = sum_p gbar_p n_bp with
  //   dvar/dk_p  = 2 (k_p - m)/N
  //   dskew/dk_p = 3[(k_p - m)^2 - mu2] mu2^-3/2 / N - 3 mu3 mu2^-5/2 (k_p - m)/N
  std::vector<double> Gb(S);
  const double i32 = 1.0 / (mu2 * std::sqrt(mu2));
  const double i52 = i32 / mu2;
  for (int b = 0; b < S; ++b) {
    const double S1 = sm[4 * b], S2 = sm[4 * b + 1], T = sm[4 * b + 2], Nb = sm[4 * b + 3];
    const double c1 = S1 - m1 * Nb;                             // sum (k-m) n
    const double c2 = S2 - 2.0 * m1 * S1 + m1 * m1 * Nb;        // sum (k-m)^2 n
    const double gv = 2.0 * c1 / N;
    const double gs = 3.0 * (c2 - mu2 * Nb) * i32 / N - 3.0 * mu3 * i52 * c1 / N;
    Gb[b] = w_var * gv + w_skew * gs + T;
  }
  const double Hs = Q;   // var and skew are shift invariant: their H is 0
  for (int j = 0; j < 5; ++j) {
    double acc = 0.0;
    for (int b = 0; b < S; ++b) acc += dA[j * S + b] * Gb[b];
    grad[j] = acc - dC[j] * Hs;
  }
  if (G)
    for (int b = 0; b < S; ++b) G[b] = Gb[b];
  if (H) *H = Hs;
}

// Adjoint sums -> gradients (host FP64 assembly).  Synchronises.
// With kappa (non-NULL) the same launch also writes the FP32 map and its
// block sums, and the moment pass gives moments and PDF
// (ufc_kappa_stats_backward).
ufc_status run_kappa_backward_ex(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                 const double* A, double C, double w_var, double w_skew,
                                 const float* g, const double* dA, const double* dC,
                                 double* grad, double* G, double* H, float* kappa, double lo,
                                 double hi, int nbins, double* moments, int64_t* pdf) {
  ufc_status s = check_kappa_args(c, counts, S, nside, A, C);
  if (s) return s;
  if (!grad) return set_err(c, UFC_ERR_ARG, "grad_theta is NULL");
  if (!dA || !dC) return set_err(c, UFC_ERR_ARG, "dA and dC are required");
  const int npix = 12 * nside * nside;
  Coef cf;
  make_coef(A, C, S, npix, cf);
  std::vector<double> sm(4 * (size_t)S + 4);
  s = adjoint_sums(c, counts, S, nside, cf, nullptr, g, kappa, lo, hi, nbins, moments, pdf,
                   sm.data());
  if (s) return s;
  grad_from_sums(sm.data(), S, npix, w_var, w_skew, dA, dC, grad, G, H);
  return UFC_OK;
}

// ---- subvolume partial sums (Sec. 2.4) --------------------------------------
ufc_status run_kappa_partial(ufc_ctx* c, const int32_t* counts, int S, int nside,
                             const double* A, double* partial) {
  ufc_status s = check_kappa_args(c, counts, S, nside, A, 0.0);
  if (s) return s;
  if (!partial) return set_err(c, UFC_ERR_ARG, "partial_dev is NULL");
  if ((reinterpret_cast<uintptr_t>(counts) & 15) || (reinterpret_cast<uintptr_t>(partial) & 15))
    return set_err(c, UFC_ERR_ARG, "counts_dev and partial_dev must be 16-byte aligned");
  const int npix = 12 * nside * nside;
  Coef cf;
  make_coef(A, 0.0, S, npix, cf);
  {
    ProfScope ps_(c, "k_kappa_partial");
    k_kappa_partial<<<kappa_fwd_grid(c), kKV, 0, c->stream>>>(counts, cf, partial);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

static ufc_status check_partial_args(ufc_ctx* c, const double* partial, int nside, double C) {
  if (!partial) return set_err(c, UFC_ERR_ARG, "partial_dev is NULL");
  if (reinterpret_cast<uintptr_t>(partial) & 15)
    return set_err(c, UFC_ERR_ARG, "partial_dev must be 16-byte aligned");
  if (nside < 1 || nside > UFC_MAX_NSIDE || (nside & (nside - 1)))
    return set_err(c, UFC_ERR_ARG, "nside must be a power of two in [1,%d]", UFC_MAX_NSIDE);
  if (!std::isfinite(C)) return set_err(c, UFC_ERR_ARG, "C is not finite");
  return UFC_OK;
}

ufc_status run_kappa_stats_partial(ufc_ctx* c, const double* partial, int nside, double C,
                                   double lo, double hi, int nbins, float* kappa,
                                   double* moments, int64_t* pdf) {
  ufc_status s = check_partial_args(c, partial, nside, C);
  if (s) return s;
  if (!kappa || !moments || !pdf)
    return set_err(c, UFC_ERR_ARG, "kappa_dev, moments_dev and pdf_dev are required");
  if (reinterpret_cast<uintptr_t>(kappa) & 15)
    return set_err(c, UFC_ERR_ARG, "kappa_dev must be 16-byte aligned");
  if (nbins < 1 || nbins > kMaxBins)
    return set_err(c, UFC_ERR_ARG, "nbins must be in [1,%d]", kMaxBins);
  if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
    return set_err(c, UFC_ERR_ARG, "PDF range needs finite lo < hi");
  const int npix = 12 * nside * nside;
  const int grid = kappa_fwd_grid(c), mgrid = 2 * c->num_sms;
  double* ksum = (double*)ws_get(c, kSlotPartials, (size_t)(grid + 3 * mgrid) * 8);
  if (!ksum) return UFC_ERR_ALLOC;
  const float ch = (float)C, cl = (float)(C - (double)ch);
  {
    ProfScope ps_(c, "k_kappa_finish");
    k_kappa_finish<<<grid, kKV, 0, c->stream>>>(partial, ch, cl, npix, kappa, ksum);
  }
  UFC_CUDA(c, cudaGetLastError());
  return launch_moments(c, kappa, npix, ksum, grid, lo, hi, nbins, ksum + grid, mgrid, moments,
                        pdf, true);
}

ufc_status run_kappa_adjoint_sums(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                  const double* partial, double C, const float* g, float* kappa,
                                  double lo, double hi, int nbins, double* moments, int64_t* pdf,
                                  double* sums) {
  ufc_status s = check_partial_args(c, partial, nside, C);
  if (s) return s;
  if (!counts) return set_err(c, UFC_ERR_ARG, "counts_dev is NULL");
  if (S < 1 || S > kMaxShells) return set_err(c, UFC_ERR_ARG, "nshell must be in [1,%d]", kMaxShells);
  if ((int64_t)S * 12 * nside * nside >= (1ll << 31))
    return set_err(c, UFC_ERR_ARG, "nshell * 12 nside^2 must be < 2^31");
  if (!sums) return set_err(c, UFC_ERR_ARG, "sums is NULL");
  const int npix = 12 * nside * nside;
  std::vector<double> zeros(S, 0.0);
  Coef cf;
  make_coef(zeros.data(), C, S, npix, cf);   // A unused: e comes from the partials
  return adjoint_sums(c, counts, S, nside, cf, partial, g, kappa, lo, hi, nbins, moments, pdf,
                      sums);
}

ufc_status run_kappa_backward(ufc_ctx* c, const int32_t* counts, int S, int nside,
                              const double* A, double C, double w_var, double w_skew,
                              const float* g, const double* dA, const double* dC,
                              double* grad, double* G, double* H) {
  return run_kappa_backward_ex(c, counts, S, nside, A, C, w_var, w_skew, g, dA, dC, grad, G, H,
                               nullptr, 0.0, 1.0, 1, nullptr, nullptr);
}

// ---- variant of ufc_kappa_stats that allocates nothing -------------------
// Its per-block partial sums live in this file-scope device array instead of
// the context workspace.  Every GPU that loads the library holds the array
// (kNoAllocScratch doubles = 32 KB) until the process exits; all calls on a
// device share it, so calls that overlap on the GPU race on it.
constexpr int kNoAllocScratch = 4096;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) the first time the variant runs there.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {};

static ufc_status noalloc_scratch(ufc_ctx* c, double** out) {
  if (c->device < 0 || c->device >= 64)
    return set_err(c, UFC_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[c->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_err(c, UFC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                     cudaGetErrorString(e));
    g_noalloc_ptr[c->device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[c->device];
  return UFC_OK;
}

ufc_status run_kappa_stats_noalloc(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                   const double* A, double C, double lo, double hi, int nbins,
                                   float* kappa, double* moments, int64_t* pdf) {
  ufc_status s = check_kappa_args(c, counts, S, nside, A, C);
  if (s) return s;
  if (!kappa || !moments || !pdf)
    return set_err(c, UFC_ERR_ARG, "the no-allocation variant needs kappa_dev, moments_dev and pdf_dev");
  if (nbins < 1 || nbins > kMaxBins)
    return set_err(c, UFC_ERR_ARG, "nbins must be in [1,%d]", kMaxBins);
  if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
    return set_err(c, UFC_ERR_ARG, "PDF range needs finite lo < hi");
  if (reinterpret_cast<uintptr_t>(counts) & 15)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 16-byte aligned");
  const int npix = 12 * nside * nside;
  const int grid = kappa_fwd_grid(c);
  const int mgrid = 2 * c->num_sms;
  if (grid + 3 * mgrid > kNoAllocScratch)
    return set_err(c, UFC_ERR_CAPACITY,
                   "scratch needs %d doubles, the fixed array holds %d", grid + 3 * mgrid,
                   kNoAllocScratch);
  double* ksum = nullptr;
  s = noalloc_scratch(c, &ksum);
  if (s) return s;
  double* mpart = ksum + grid;   // every slot is written before it is read
  Coef cf;
  make_coef(A, C, S, npix, cf);
  s = launch_kappa_fwd(c, counts, cf, kappa, ksum, grid);
  if (s) return s;
  // (no kernel-timing records here: recording them may allocate)
  return launch_moments(c, kappa, npix, ksum, grid, lo, hi, nbins, mpart, mgrid, moments, pdf,
                        false);
}

ufc_status run_stats_vector(ufc_ctx* c, const double* m, const int64_t* pdf, int nbins,
                            double* v) {
  if (!m || !pdf || !v || nbins < 1 || nbins > kMaxBins)
    return set_err(c, UFC_ERR_ARG, "stats_vector: bad arguments");
  {
    ProfScope ps_(c, "k_stats_vector");
    k_stats_vector<<<1, 256, 0, c->stream>>>(m, (const unsigned long long*)pdf, nbins, v);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

ufc_status run_welford_update(ufc_ctx* c, const double* v, int nvec, int d, double* st) {
  if (!v || !st || nvec < 0 || d < 1 || d > 8192)
    return set_err(c, UFC_ERR_ARG, "welford_update: bad arguments");
  if (nvec == 0) return UFC_OK;
  const int smem = 2 * welford_run(d) * d * 8;   // up to 128 KB at d = 8192
  UFC_CUDA(c, cudaFuncSetAttribute(k_welford_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem));
  {
    ProfScope ps_(c, "k_welford_update");
    k_welford_update<<<1, 1024, smem, c->stream>>>(v, nvec, d, st);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}
ufc_status run_welford_merge(ufc_ctx* c, double* a, const double* b, int d) {
  if (!a || !b || d < 1 || d > 8192) return set_err(c, UFC_ERR_ARG, "welford_merge: bad arguments");
  {
    ProfScope ps_(c, "k_welford_merge");
    k_welford_merge<<<1, 1024, 0, c->stream>>>(a, b, d);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}
ufc_status run_welford_finalize(ufc_ctx* c, const double* st, int d, int ddof, double* mean,
                                double* cov, double* corr) {
  if (!st || !mean || !cov || !corr || d < 1 || d > 8192 || ddof < 0)
    return set_err(c, UFC_ERR_ARG, "welford_finalize: bad arguments");
  {
    ProfScope ps_(c, "k_welford_final");
    k_welford_final<<<1, 1024, 0, c->stream>>>(st, d, ddof, mean, cov, corr);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

// ---- persistent batched call: host side ------------------------------------
ufc_status batch_geometry(ufc_ctx* c, const double* chi, int nshell, const ufc_box* boxes,
                          int nbox, ShellTable& st, BoxGeom* bg);
void batch_bands(int nside, float smax, Bands& bd);

// Workspace of the persistent batch kernel: per realisation a count map, a
// kappa map and the partial sums of the serial grids (256-byte aligned
// pieces), and the descriptors.
static size_t batch_map_stride(int S, int nside) {
  return ((size_t)S * 12 * nside * nside * 4 + 255) / 256 * 256;
}
void batch_persistent_bytes(const ufc_ctx* c, int nreal, int nbox, int S, int nside,
                            size_t* maps, size_t* desc) {
  const size_t npix = 12ull * nside * nside;
  const size_t kap_b = (npix * 4 + 255) / 256 * 256;
  const size_t part_b = ((size_t)(8 * c->num_sms + 3 * 2 * c->num_sms) * 8 + 255) / 256 * 256;
  *maps = (batch_map_stride(S, nside) + kap_b + part_b) * nreal;
  *desc = ((size_t)nreal * nbox * sizeof(BatchItem) + 255) / 256 * 256 +
          ((size_t)nreal * sizeof(Coef) + 255) / 256 * 256 + ((size_t)nreal * 4 + 255) / 256 * 256 +
          16 + (size_t)nreal * 4 + 256;
}

struct BatchLaunch {
  BatchArgs ba;
  ShellTable st;
  Bands bd;
  PdfParam pp;
  size_t zero_maps;          // bytes of count maps to clear at each launch
  size_t q_off, q_bytes;     // queue counters in the descriptor buffer
  int grid, smem;
};

// Host set-up of a persistent batched call: geometry, descriptors uploaded
// into `desc` (synchronises the context stream; never under stream capture),
// launch arguments kept in the context.
ufc_status batch_persistent_prepare(ufc_ctx* c, int nreal, int nbox, const float* const* xyz,
                                    const int64_t* n, const ufc_box* boxes, const double* chi,
                                    int S, int nside, const double* A, const double* C, double lo,
                                    double hi, int nbins, double* moments, int64_t* pdf,
                                    double* stats, double* state, char* maps, char* desc) {
  const int npix = 12 * nside * nside;
  const int nitems = nreal * nbox;
  const int chunk = c->batch_chunk > 0 ? c->batch_chunk : 8192;
  const int bps = c->batch_blocks_per_sm > 0 ? c->batch_blocks_per_sm : 2;
  std::vector<BoxGeom> bg(nbox);
  BatchLaunch L;
  std::memset(&L, 0, sizeof L);
  std::vector<BatchItem> items(nitems);
  std::vector<int32_t> ntask_r(nreal, 0);
  float smax = 0.f;
  int64_t task = 0;
  for (int r = 0; r < nreal; ++r) {
    ufc_status s = batch_geometry(c, chi, S, boxes + (size_t)r * nbox, nbox, L.st, bg.data());
    if (s) return s;
    for (int k = 0; k < nbox; ++k) {
      const size_t i = (size_t)r * nbox + k;
      BatchItem& it = items[i];
      const BoxGeom& g = bg[k];
      if (n[i] < 0) return set_err(c, UFC_ERR_ARG, "n[%zu] < 0", i);
      if (n[i] > 0 && !xyz[i]) return set_err(c, UFC_ERR_ARG, "xyz[%zu] is NULL", i);
      smax = std::max(smax, g.smax);
      it.xyz = xyz[i];
      it.n = n[i];
      it.task0 = task;
      it.real = r;
      it.shell_lo = g.shell_lo;
      it.shell_hi = g.shell_hi;
      for (int ax = 0; ax < 3; ++ax) {
        it.shf[ax] = g.shf[ax][0];
        it.shlo[ax] = g.shlo[ax][0];
        it.sh64[ax] = g.sh64[ax][0];
      }
      const int64_t nt = std::max<int64_t>(1, (it.n + chunk - 1) / chunk);   // empty: one task
      task += nt;
      ntask_r[r] += (int32_t)nt;
    }
  }
  batch_bands(nside, smax, L.bd);        // the bands of the largest shift of all the boxes
  std::vector<Coef> coef(nreal);
  for (int r = 0; r < nreal; ++r) make_coef(A + (size_t)r * S, C[r], S, npix, coef[r]);
  const size_t o_coef = ((size_t)nitems * sizeof(BatchItem) + 255) / 256 * 256;
  const size_t o_nt = o_coef + ((size_t)nreal * sizeof(Coef) + 255) / 256 * 256;
  const size_t o_q = o_nt + ((size_t)nreal * 4 + 255) / 256 * 256;
  std::vector<char> host(o_q);
  std::memcpy(host.data(), items.data(), (size_t)nitems * sizeof(BatchItem));
  std::memcpy(host.data() + o_coef, coef.data(), (size_t)nreal * sizeof(Coef));
  std::memcpy(host.data() + o_nt, ntask_r.data(), (size_t)nreal * 4);
  UFC_CUDA(c, cudaMemcpyAsync(desc, host.data(), host.size(), cudaMemcpyHostToDevice, c->stream));
  UFC_CUDA(c, cudaStreamSynchronize(c->stream));   // (host staging leaves scope)
  const int gk = kappa_fwd_grid(c), gm = 2 * c->num_sms;
  const size_t map_b = batch_map_stride(S, nside);
  const size_t kap_b = ((size_t)npix * 4 + 255) / 256 * 256;
  BatchArgs& ba = L.ba;
  ba.items = reinterpret_cast<const BatchItem*>(desc);
  ba.nitems = nitems;
  ba.chunk = chunk;
  ba.ntasks = task;
  ba.coef = reinterpret_cast<const Coef*>(desc + o_coef);
  ba.ntask_r = reinterpret_cast<const int32_t*>(desc + o_nt);
  ba.nreal = nreal;
  ba.S = S;
  ba.N = nside;
  ba.npix = npix;
  ba.counts = reinterpret_cast<int32_t*>(maps);
  ba.kappa = reinterpret_cast<float*>(maps + map_b * nreal);
  ba.ksum = reinterpret_cast<double*>(maps + (map_b + kap_b) * nreal);
  ba.mpart = ba.ksum + (size_t)gk * nreal;
  ba.gk = gk;
  ba.gm = gm;
  ba.moments = moments;
  ba.pdf = pdf;
  ba.stats = stats;
  ba.state = state;
  ba.nbins = nbins;
  ba.d = 6 + nbins;
  ba.queue = reinterpret_cast<unsigned long long*>(desc + o_q);
  ba.done = reinterpret_cast<unsigned int*>(desc + o_q + 16);
  if (map_b != (size_t)S * npix * 4)      // maps are indexed as [nreal][S][npix]
    return set_err(c, UFC_ERR_UNSUPPORTED, "persistent batch: map size not a multiple of 256 B");
  L.pp = make_pdf_param(lo, hi, nbins);
  L.zero_maps = map_b * nreal;
  L.q_off = o_q;
  L.q_bytes = 16 + (size_t)nreal * 4;
  L.grid = std::min(bps, 2) * c->num_sms;
  L.smem = std::max((nbins + 3) * 4, 2 * welford_run(6 + nbins) * (6 + nbins) * 8);
  c->batch_launch.resize(sizeof L);
  std::memcpy(c->batch_launch.data(), &L, sizeof L);
  // (static plus dynamic shared memory may pass the 48 KB default)
  UFC_CUDA(c, cudaFuncSetAttribute(k_batch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   L.smem));
  return UFC_OK;
}

// The launch itself (capturable): clear the maps and the queue, run the kernel.
ufc_status batch_persistent_enqueue(ufc_ctx* c, char* maps, char* desc) {
  if (c->batch_launch.size() != sizeof(BatchLaunch))
    return set_err(c, UFC_ERR_ARG, "persistent batch: no prepared launch");
  BatchLaunch L;
  std::memcpy(&L, c->batch_launch.data(), sizeof L);
  UFC_CUDA(c, cudaMemsetAsync(maps, 0, L.zero_maps, c->stream));
  UFC_CUDA(c, cudaMemsetAsync(desc + L.q_off, 0, L.q_bytes, c->stream));
  {
    ProfScope ps_(c, "k_batch_persistent");
    k_batch_persistent<<<L.grid, kBT, L.smem, c->stream>>>(L.ba, L.st, L.bd, L.pp);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

}  // namespace ufc

