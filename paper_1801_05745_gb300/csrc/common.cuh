// Internal definitions shared by the CUDA translation units of
// libufalcon_gb300.so.  Nothing here is part of the C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ufalcon.h"

namespace ufc {

constexpr int kMaxShells = UFC_MAX_SHELLS;
constexpr int kMaxImg1D = 2 * UFC_MAX_REPLICATE + 1;
constexpr int kMaxBoxes = 16;

// Key sentinels of ufc_keys.
constexpr int32_t kKeyOutside = -1;
constexpr int32_t kKeyInvalid = -2;
// Internal key of an undecided particle in the FP32 stage.
constexpr int32_t kKeyUndecided = -3;

// Geometry of one box as the key kernels see it.  The FP64 image shifts
// shift = fl(fl(i L) - o) are split into an FP32 high part and an FP32
// remainder for the FP32 and double-float stages.
struct BoxGeom {
  double sh64[3][kMaxImg1D];
  float shf[3][kMaxImg1D];
  float shlo[3][kMaxImg1D];
  int32_t shell_lo, shell_hi;   // owned shells [lo, hi)
  int32_t R;                    // image layers
  int32_t nimg;                 // (2R+1)^3
  float smax;                   // max |shift| over images and axes
  float pad_;
};

// Shell edges and FP32 decision bands.  An FP32 squared radius r2f below
// lo2[e] is certainly below chi_e (in the FP64 procedure), one at or above
// hi2[e] certainly at or above it.
struct ShellTable {
  double chi64[kMaxShells + 1];
  float chih[kMaxShells + 1];   // chi64 as double-float (hi + lo)
  float chil[kMaxShells + 1];
  float lo2[kMaxShells + 1];
  float hi2[kMaxShells + 1];
  int32_t nshell;
  int32_t pad_;
};

// FP32-stage bands, computed on the host from the error analysis of the
// FP32 operations (u = 2^-24), twice the analysed bound.
struct Bands {
  float z_eq;       // |z| <= z_eq  => equatorial belt for certain
  float z_cap;      // |z| >  z_cap => polar cap for certain
  float eq;         // 1/2 - (absolute band of the equatorial edge coordinates) - 2^-23
  float cap;        // 1/2 - (absolute band of the cap edge coordinates) - 2^-23
  float eq_d;       // 1/2 - eq: least distance of a certain equatorial edge coordinate
                    // from the nearest integer
  float cap_d;      // 1/2 - cap, the same for the cap edge coordinates
  float ip_per_ir;  // band of the in-ring coordinate t*ir, per unit of ir
  float r2_min;     // below this squared radius: undecided
  float axy_min;    // max(|dx|,|dy|) below this: undecided
  float z_eq2;      // dz^2 <= z_eq2 r2  => equatorial belt for certain
  float z_cap2;     // dz^2 >  z_cap2 r2 => polar cap for certain
  // constants of the pixel arithmetic for the map's N, read as kernel
  // parameters instead of being recomputed per group
  float fN;         // N
  float n75;        // 3N/4 (exact)
  float c0;         // 1/2 when N = 1, else 0
  int32_t nhalf;    // N >> 1
  int32_t ring0;    // 2 N (N - 1), the first pixel of the belt
  int32_t four_n;   // 4 N
  int32_t eight_n;  // 8 N
  int32_t npix;     // 12 N^2
};

struct GeomAll {
  int32_t nside;
  int32_t npix;       // 12 nside^2
  int32_t nbox;
  int32_t pad_;
  BoxGeom box[kMaxBoxes];
};

// Device-side counters of a binning call.
struct BinCounters {
  unsigned long long invalid;
  unsigned long long keyed;
  unsigned long long refined;   // entered the double-float stage
  unsigned long long exact;     // entered the FP64 stage
  unsigned long long q1;        // entries in queue 1
  unsigned long long q2;        // entries in queue 2
  unsigned long long dense;     // keys written by the compaction stage
  unsigned long long ntiles;    // tiles of the second scatter pass
  unsigned long long range;     // adjoint inputs outside the fixed-point range
  unsigned long long ovf;       // images marked for the exact pass (queue 1 was full)
  // bounded device waits that ran out: last, so that a binning call's reset
  // (everything before it) keeps it until ufc_synchronize reports it
  unsigned long long timeouts;
};

// ---- index checks of checked builds ----------------------------------------
// A build with -DUFC_CHECKED tests computed indices at the sites marked
// UFC_IDX_OK(index, bound, site): a failed test counts in its translation
// unit's record, which keeps the first failure's site, index and bound, and
// the access is skipped, so the kernel runs to its end; ufc_synchronize
// reports the failure (UFC_ERR_INTERNAL).  Other builds compile the tests
// away (UFC_IDX_OK is the constant true).  The record is one per device and
// translation unit, shared by the contexts on that device.
struct CheckRec {
  unsigned long long count;
  long long site, index, bound;
};
static __device__ CheckRec g_check;
__device__ __forceinline__ bool check_idx(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_check.count, 1ull) == 0ull) {
    g_check.site = site;
    g_check.index = i;
    g_check.bound = n;
  }
  return false;
}
#ifdef UFC_CHECKED
#define UFC_IDX_OK(i, n, site) (::ufc::check_idx((long long)(i), (long long)(n), (site)))
#else
#define UFC_IDX_OK(i, n, site) true
#endif
// Reads this translation unit's record into *out and clears it, on stream s
// (the caller synchronises).
static inline cudaError_t take_check_rec(CheckRec* out, cudaStream_t s) {
  static const CheckRec zero{};
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_check, sizeof(CheckRec), 0,
                                            cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbolAsync(g_check, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
}

// Queue entry of an undecided particle image: box (4 bits), image (13 bits),
// particle index (47 bits).
__host__ __device__ inline uint64_t qpack(int box, int img, int64_t p) {
  return (uint64_t(box) << 60) | (uint64_t(img) << 47) | uint64_t(p);
}
__host__ __device__ inline int qbox(uint64_t e) { return int(e >> 60); }
__host__ __device__ inline int qimg(uint64_t e) { return int((e >> 47) & 0x1FFF); }
__host__ __device__ inline int64_t qidx(uint64_t e) { return int64_t(e & ((1ull << 47) - 1)); }

}  // namespace ufc
