// Particle -> (shell, RING pixel) keys and per-shell count maps (Eq. 5,
// Eq. 8 and the HEALPix pixelisation of Sec. 2.4).
//
// Pipeline of one binning call:
//   fast stage  k_fast    : one pass over the particles (FP32 arithmetic);
//                           decided keys go to the output, undecided
//                           particle images to queue 1.
//   refine stage k_refine : double-float over queue 1; undecided to queue 2.
//   exact stage k_exact   : the FP64 procedure over queue 2.
// Outputs (mode):
//   KEYS   : int32 key per particle (ufc_keys).
//   DIRECT : atomicAdd into the count map (maps that sit in L2).
//   DENSE  : keys packed as (bucket << 15 | offset) with bucket = shell *
//            nblk + pix / 24576, appended per warp to a dense array while a
//            shared-memory histogram counts buckets; then two scatter passes
//            (by bucket group, then by bucket) and a shared-memory histogram
//            per bucket that writes each 24576-pixel block of the count map
//            once.  No global atomics on the count map.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstddef>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "pixel.cuh"

namespace ufc {

enum Mode { kModeKeys = 0, kModeDirect = 1, kModeDense = 2 };

constexpr int kBlockPix = 24576;        // pixels per count-map block (96 KB of u32)
constexpr int kOffBits = 15;            // offset bits in a dense key
constexpr uint32_t kSentinel = 0xFFFFFFFFu;
constexpr int kChunk = 2048;            // dense keys reserved per warp at a time
constexpr int kGroupBits = 8;           // buckets per group = 256
constexpr int kSmemHistMax = 45056;     // buckets counted in shared memory
constexpr int kFastThreads = 512;

struct KeyOut {
  int32_t* keys;               // KEYS
  int32_t* counts;             // DIRECT
  uint32_t* dense;             // DENSE
  unsigned long long* dense_count;
  uint32_t* hist;              // DENSE: global bucket histogram
  int64_t dense_cap;
  int32_t nblk;                // blocks per shell (DENSE)
  int32_t nbuckets;
  int32_t shell0;              // DENSE: first shell of the call's window; buckets
                               // count blocks from shell0 * nblk
  int32_t smem_hist;           // 1: histogram in shared memory
  int64_t ncell;               // cells of the count map (checked builds' bound)
};

struct Queues {
  uint64_t* q1;
  uint64_t* q2;
  int64_t cap1, cap2;
  BinCounters* cnt;
  uint32_t* ovf;        // one bit per particle of the boxes without images
  int64_t ovf_base;     // first bit of the launch's box
};

// ---------------------------------------------------------------- emission --
struct WarpChunk {
  int64_t base;   // start of the warp's current chunk (-1: none)
  int32_t fill;
  bool fits;      // the whole chunk lies below the capacity (always, with the
                  // workspace's sizes; a chunk that did not would be dropped)
};

__device__ __forceinline__ uint32_t dense_key(int32_t key, int32_t npix, const KeyOut& o) {
  int32_t b = key / npix;
  int32_t pix = key - b * npix;
  int32_t blk = pix / kBlockPix;
  return (uint32_t((b - o.shell0) * o.nblk + blk) << kOffBits) | uint32_t(pix - blk * kBlockPix);
}

// Appends the keys of lanes with `want` to the warp's chunk of the dense
// array (all 32 lanes call this together).
__device__ __forceinline__ void dense_append(WarpChunk& wc, bool want, uint32_t v,
                                             const KeyOut& o) {
  const unsigned full = 0xFFFFFFFFu;
  unsigned m = __ballot_sync(full, want);
  if (m == 0) return;
  int lane = threadIdx.x & 31;
  int cnt = __popc(m);
  int rank = __popc(m & ((1u << lane) - 1u));
  if (wc.base < 0) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(o.dense_count, (unsigned long long)kChunk);
    wc.base = (int64_t)__shfl_sync(full, b, 0);
    wc.fill = 0;
    wc.fits = wc.base + kChunk <= o.dense_cap;
  }
  int room = kChunk - wc.fill;
  if (want && rank < room && wc.fits) o.dense[wc.base + (wc.fill + rank)] = v;
  if (cnt >= room) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(o.dense_count, (unsigned long long)kChunk);
    int64_t nb = (int64_t)__shfl_sync(full, b, 0);
    const bool nfits = nb + kChunk <= o.dense_cap;
    if (want && rank >= room && nfits) o.dense[nb + (rank - room)] = v;
    wc.base = nb;
    wc.fits = nfits;
    wc.fill = cnt - room;
  } else {
    wc.fill += cnt;
  }
}

__device__ __forceinline__ void dense_close(WarpChunk& wc, const KeyOut& o) {
  if (wc.base < 0) return;
  int lane = threadIdx.x & 31;
  for (int i = wc.fill + lane; i < kChunk; i += 32)
    if (wc.base + i < o.dense_cap) o.dense[wc.base + i] = kSentinel;
}

// Warp-aggregated push of undecided entries into per-warp chunks of
// kQChunk queue slots (one atomic per chunk, not per push); returns false for
// lanes whose entry did not fit (they resolve it themselves).  Unused slots
// of a warp's last chunk hold kQEmpty.
constexpr int kQChunk = 256;
constexpr uint64_t kQEmpty = ~0ull;
struct QChunk {
  int64_t base;   // -1: none
  int32_t fill;
};

// `entry()` gives the value; it is evaluated only by lanes that push.
template <class F>
__device__ __forceinline__ bool queue_push_f(QChunk& qc, bool want, F entry, uint64_t* q,
                                             int64_t cap, unsigned long long* count) {
  const unsigned full = 0xFFFFFFFFu;
  const unsigned m = __ballot_sync(full, want);
  if (m == 0) return true;
  const int lane = threadIdx.x & 31;
  const int cnt = __popc(m);
  const int rank = __popc(m & ((1u << lane) - 1u));
  if (qc.base < 0) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(count, (unsigned long long)kQChunk);
    qc.base = (int64_t)__shfl_sync(full, b, 0);
    qc.fill = 0;
  }
  const int room = kQChunk - qc.fill;
  int64_t idx;
  if (rank < room) {
    idx = qc.base + qc.fill + rank;
  } else {
    idx = -1;
  }
  if (cnt >= room) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(count, (unsigned long long)kQChunk);
    const int64_t nb = (int64_t)__shfl_sync(full, b, 0);
    if (rank >= room) idx = nb + (rank - room);
    qc.base = nb;
    qc.fill = cnt - room;
  } else {
    qc.fill += cnt;
  }
  if (!want) return true;
  if (idx < cap) { q[idx] = entry(); return true; }
  return false;
}
__device__ __forceinline__ bool queue_push(QChunk& qc, bool want, uint64_t e, uint64_t* q,
                                           int64_t cap, unsigned long long* count) {
  return queue_push_f(qc, want, [e]() { return e; }, q, cap, count);
}

// queue_push_f whose entries that find the queue full set their particle's
// bit (base + particle index) in the overflow bitmap instead.
template <class F>
__device__ __forceinline__ void queue_push_mark(QChunk& qc, bool want, F entry, uint64_t* q,
                                                int64_t cap, unsigned long long* count,
                                                uint32_t* ovf, int64_t ovf_base,
                                                unsigned long long* flag) {
  const unsigned full = 0xFFFFFFFFu;
  const unsigned m = __ballot_sync(full, want);
  if (m == 0) return;
  const int lane = threadIdx.x & 31;
  const int cnt = __popc(m);
  const int rank = __popc(m & ((1u << lane) - 1u));
  if (qc.base < 0) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(count, (unsigned long long)kQChunk);
    qc.base = (int64_t)__shfl_sync(full, b, 0);
    qc.fill = 0;
  }
  const int room = kQChunk - qc.fill;
  int64_t idx = rank < room ? qc.base + qc.fill + rank : -1;
  if (cnt >= room) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(count, (unsigned long long)kQChunk);
    const int64_t nb = (int64_t)__shfl_sync(full, b, 0);
    if (rank >= room) idx = nb + (rank - room);
    qc.base = nb;
    qc.fill = cnt - room;
  } else {
    qc.fill += cnt;
  }
  if (!want) return;
  const uint64_t e = entry();
  if (idx < cap) {
    q[idx] = e;
  } else {
    const uint64_t bit = uint64_t(ovf_base) + uint64_t(qidx(e));
    atomicOr(ovf + (bit >> 5), 1u << (bit & 31u));
    *flag = 1ull;
  }
}

// Marks the unused slots of the warp's last queue chunk.
__device__ __forceinline__ void queue_close(QChunk& qc, uint64_t* q, int64_t cap) {
  if (qc.base < 0) return;
  const int lane = threadIdx.x & 31;
  for (int i = qc.fill + lane; i < kQChunk; i += 32)
    if (qc.base + i < cap) q[qc.base + i] = kQEmpty;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

// ----------------------------------------------------------- fast stage ----
// Shell lookup table over r^2.  Bin i holds the r2 values whose FP32
// v = fminf(r2 * scale, kLut - 1) rounds to i; its low 15 bits count the
// edges e certainly at or below every such r2 (hi2[e] <= the bin's lowest
// possible r2), and bit 15 is set unless the next edge is certainly above
// every such r2 (lo2[e0] > the bin's highest possible r2).  A clean bin
// gives the shell with one load; the others scan the edges (exact).
constexpr int kLutBits = 13;
constexpr int kLut = 1 << kLutBits;
constexpr uint16_t kLutScan = 0x8000;

struct FastShared {
  float lo2[kMaxShells + 2], hi2[kMaxShells + 2];
  float shf[3][kMaxImg1D], shlo[3][kMaxImg1D];
  uint16_t lut[kLut];
};

// Shell of r2 (finite, >= 0) among the box's shells [lo, hi): -1 outside,
// -2 undecided.
__device__ __forceinline__ int32_t shell_lut(const FastShared& fs, int32_t lo, int32_t hi,
                                             float lut_scale, float r2) {
  const float v = fminf(r2 * lut_scale, float(kLut - 1));
  const int bin = __float_as_int(v + 8388608.0f) - 0x4B000000;   // round(v), exact
  const uint32_t e = fs.lut[bin];
  int a = int(e & 0x7FFFu) - 1;
  if (e & kLutScan) {
    for (;;) {                                  // ends at the +inf sentinel
      if (r2 < fs.lo2[a + 1]) break;            // certainly below edge a+1
      if (r2 < fs.hi2[a + 1]) return -2;        // inside edge a+1's band
      ++a;
    }
  }
  return (a >= lo && a < hi) ? a : -1;
}

struct FastCtx {
  WarpChunk wc;
  QChunk qc;
  unsigned long long n_invalid, n_keyed;
};

// All images of one particle (warp-collective: every lane calls it).
template <int MODE>
__device__ __forceinline__ void fast_particle(bool have, float x, float y, float zc, int64_t p,
                                              int32_t box_id, const BoxGeom& bg,
                                              const FastShared& fs, float lut_scale,
                                              const ShellTable& st, const Bands& bd, int32_t N,
                                              int32_t npix, const KeyOut& o, const Queues& qs,
                                              uint32_t* hist_s, FastCtx& fc) {
  const int lo = bg.shell_lo, hi = bg.shell_hi;
  const int n1 = 2 * bg.R + 1;
  const bool finite = have && isfinite(x) && isfinite(y) && isfinite(zc);
  if (have && !finite) ++fc.n_invalid;
  int ii = 0, jj = 0, kk = 0;                   // image (ii, jj, kk), img = (ii n1 + jj) n1 + kk
  for (int img = 0; img < bg.nimg; ++img) {
    if (img) {
      if (++kk == n1) { kk = 0; if (++jj == n1) { jj = 0; ++ii; } }
    }
    int32_t key = kKeyOutside;
    uint32_t dkey = 0u;
    if (finite) {
      const float dx = (x + fs.shf[0][ii]) + fs.shlo[0][ii];
      const float dy = (y + fs.shf[1][jj]) + fs.shlo[1][jj];
      const float dz = (zc + fs.shf[2][kk]) + fs.shlo[2][kk];
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      if (!(r2 >= bd.r2_min)) {
        key = kKeyUndecided;
      } else {
        const int32_t b = shell_lut(fs, lo, hi, lut_scale, r2);
        if (b == -2) {
          key = kKeyUndecided;
        } else if (b >= 0) {
          const int32_t pix = pixel_fast(N, bd, dx, dy, dz, r2);
          key = (pix == kKeyUndecided) ? kKeyUndecided : b * npix + pix;
          if (MODE == kModeDense && pix != kKeyUndecided) {
            const uint32_t blk = uint32_t(pix >> 13) / 3u;       // pix / 24576
            dkey = ((uint32_t(b - o.shell0) * uint32_t(o.nblk) + blk) << kOffBits) |
                   (uint32_t(pix) - blk * uint32_t(kBlockPix));
          }
        }
      }
    }
    const bool und = key == kKeyUndecided;
    if (!queue_push(fc.qc, und, qpack(box_id, img, p), qs.q1, qs.cap1, &qs.cnt->q1)) {
      // queue full: resolve with the FP64 procedure here
      key = key_exact(st, lo, hi, N, npix, x, y, zc, bg.sh64[0][ii], bg.sh64[1][jj],
                      bg.sh64[2][kk]);
      if (key == kKeyInvalid) ++fc.n_invalid;
      if (MODE == kModeDense && key >= 0) dkey = dense_key(key, npix, o);
    }
    if (MODE == kModeKeys) {
      if (have) o.keys[p] = finite ? key : kKeyInvalid;
    } else if (MODE == kModeDirect) {
      if (key >= 0 && UFC_IDX_OK(key, o.ncell, 2)) atomicAdd(o.counts + key, 1);
    } else {
      if (key >= 0) {
        const uint32_t bucket = dkey >> kOffBits;
        if (UFC_IDX_OK(bucket, o.nbuckets, 1)) {
          if (o.smem_hist) atomicAdd(hist_s + bucket, 1u);
          else atomicAdd(o.hist + bucket, 1u);
        }
      }
      dense_append(fc.wc, key >= 0, dkey, o);
    }
    fc.n_keyed += key >= 0;
  }
}

__device__ __forceinline__ void fast_init_shared(FastShared& fs, const BoxGeom& bg,
                                                 const ShellTable& st, const uint16_t* lut) {
  for (int i = threadIdx.x; i <= st.nshell; i += blockDim.x) {
    fs.lo2[i] = st.lo2[i];
    fs.hi2[i] = st.hi2[i];
  }
  if (threadIdx.x == 0) {
    fs.lo2[st.nshell + 1] = INFINITY;
    fs.hi2[st.nshell + 1] = INFINITY;
  }
  for (int i = threadIdx.x; i < 3 * kMaxImg1D; i += blockDim.x) {
    fs.shf[i / kMaxImg1D][i % kMaxImg1D] = bg.shf[i / kMaxImg1D][i % kMaxImg1D];
    fs.shlo[i / kMaxImg1D][i % kMaxImg1D] = bg.shlo[i / kMaxImg1D][i % kMaxImg1D];
  }
  for (int i = threadIdx.x; i < kLut; i += blockDim.x) fs.lut[i] = lut[i];
}

template <int MODE>
__device__ __forceinline__ void fast_finish(FastCtx& fc, const KeyOut& o, const Queues& qs,
                                            uint32_t* hist_s) {
  if (MODE == kModeDense) dense_close(fc.wc, o);
  queue_close(fc.qc, qs.q1, qs.cap1);
  const unsigned long long ni = warp_sum(fc.n_invalid), nk = warp_sum(fc.n_keyed);
  if ((threadIdx.x & 31) == 0) {
    if (ni) atomicAdd(&qs.cnt->invalid, ni);
    if (nk) atomicAdd(&qs.cnt->keyed, nk);
  }
  if (MODE == kModeDense && o.smem_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < o.nbuckets; i += blockDim.x)
      if (hist_s[i]) atomicAdd(o.hist + i, hist_s[i]);
  }
}

struct LutParam { uint16_t v[kLut]; float scale; };

// Fast stage with plain per-thread loads (any 4-byte aligned input).
template <int MODE>
__global__ void __launch_bounds__(kFastThreads)
k_fast(const float* __restrict__ xyz, int64_t n, int64_t p_off, int32_t box_id, BoxGeom bg,
       ShellTable st, LutParam lp, Bands bd, int32_t N, int32_t npix, KeyOut o, Queues qs) {
  extern __shared__ uint32_t hist_s[];
  __shared__ FastShared fs;
  fast_init_shared(fs, bg, st, lp.v);
  if (MODE == kModeDense && o.smem_hist)
    for (int i = threadIdx.x; i < o.nbuckets; i += blockDim.x) hist_s[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (n + stride - 1) / stride;
  FastCtx fc{{-1, 0}, {-1, 0}, 0, 0};
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; ++it, p += stride) {
    const bool have = p < n;
    float x = 0.f, y = 0.f, zc = 0.f;
    if (have) {
      x = __ldg(xyz + 3 * p);
      y = __ldg(xyz + 3 * p + 1);
      zc = __ldg(xyz + 3 * p + 2);
    }
    fast_particle<MODE>(have, x, y, zc, p_off + p, box_id, bg, fs, lp.scale, st, bd, N, npix, o,
                        qs, hist_s, fc);
  }
  fast_finish<MODE>(fc, o, qs, hist_s);
}

// ---- bulk asynchronous copies (1-D TMA) and mbarriers ----------------------
constexpr long long kWaitLimit = 1ll << 28;   // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Self-test of the bounded wait: an mbarrier that expects one arrival which
// never comes; the wait gives up after `limit` polls and reports it like the
// fast stage does (the kernel then returns normally).
__global__ void k_wait_selftest(long long limit, unsigned long long* timeouts) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  bool ok = false;
  for (long long i = 0; i < limit && !ok; ++i) ok = mbar_try_wait(&bar, 0u);
  if (!ok) atomicAdd(timeouts, 1ull);
}

ufc_status run_wait_selftest(ufc_ctx* c, int64_t limit) {
  if (limit < 1 || limit > kWaitLimit)
    return set_err(c, UFC_ERR_ARG, "limit must be in [1, %lld]", (long long)kWaitLimit);
  BinCounters* bc = reinterpret_cast<BinCounters*>(c->counters);
  k_wait_selftest<<<1, 32, 0, c->stream>>>(limit, &bc->timeouts);
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

// The FP64 procedure for an image whose queue slot did not fit (rare); kept
// out of line so that the fast stage's register budget is not spent on it.
__device__ __noinline__ int32_t key_exact_slow(const ShellTable& st, int32_t lo, int32_t hi,
                                               int32_t N, int32_t npix, float x, float y,
                                               float zc, double shx, double shy, double shz) {
  return key_exact(st, lo, hi, N, npix, x, y, zc, shx, shy, shz);
}

// Fast stage fed by bulk copies, warp-autonomous.  Persistent blocks; a ring
// of kWStages chunks of kWChunk particles streams in by cp.async.bulk
// (16-byte aligned xyz).  Each warp owns a slice of kWPerWarp particles of
// every chunk and works through it alone, 32 particles at a time:
//   A: radius, shell (lookup table) and zone; the belt and cap particles are
//      appended, with their FP32 observer-relative coordinates, to two
//      circular pending lists of the warp in shared memory (ballots);
//   B: whenever a list holds 32 entries, the warp computes their pixels
//      together, so the pixel code always runs on full warps; keys go to the
//      dense array through the warp's chunk, bucket counts to 16-bit shared
//      counters (an overflow at 65536 is carried to the global histogram).
// A stage is free once every warp has finished A on it (the entries hold
// copies); the last warp to finish issues the copy that refills it, so the
// steady state has no block-wide barrier.  Without periodic images the
// lists carry over from chunk to chunk; an entry keeps its offset in its
// chunk and the chunk's sequence number modulo 4096, and the lists are
// drained at least every kWAgeFlush chunks.  With periodic images the lists
// are drained after every (chunk, image) pass.  Particle p of the launch is
// element p_off + p of the caller's array (chunked launches of ufc_bin_host).
constexpr int kWThreads = 768;
constexpr int kWChunk = 3840;                  // particles per chunk (45 KB)
constexpr int kWStages = 2;                    // the stage index of the ring loop is k & 1
static_assert(kWStages == 2, "the ring loop takes the stage of chunk k as k & 1");
constexpr int kWWarps = kWThreads / 32;        // 24
constexpr int kWPerWarp = kWChunk / kWWarps;   // 160
constexpr int kWGroups = kWPerWarp / 32;
constexpr int kWList = 64;                     // entries of one pending list
constexpr int kWAgeFlush = 1024;
static_assert(kWPerWarp % 32 == 0 && kWChunk <= 4096 && kMaxShells <= 256,
              "entry metadata: 8-bit shell, 12-bit offset, 12-bit chunk tag");
static_assert(kWAgeFlush < 4096, "chunk tags are 12-bit");

constexpr int kWSmemBase = kWStages * kWChunk * 12 + kWWarps * 2 * kWList * 16;   // ring + lists

// One increment of a 16-bit counter held in half of a 32-bit word; true when it wrapped the
// half, which hist16_carry then settles (the low half's carry undone, 65536 added globally).
__device__ __forceinline__ bool hist16_add(uint32_t* h32, uint32_t bucket) {
  const uint32_t shift = (bucket & 1u) << 4;
  const uint32_t old = atomicAdd(h32 + (bucket >> 1), 1u << shift);
  return ((old >> shift) & 0xFFFFu) == 0xFFFFu;
}

__device__ __forceinline__ void hist16_carry(uint32_t* h32, uint32_t* ghist, uint32_t bucket) {
  if ((bucket & 1u) == 0u) atomicSub(h32 + (bucket >> 1), 1u << 16);
  atomicAdd(ghist + bucket, 65536u);
}

template <int MODE, bool IMAGES>
__global__ void __launch_bounds__(kWThreads, 1)
k_fast_tma(const float* __restrict__ xyz, int64_t n, int64_t p_off, int32_t box_id, BoxGeom bg,
           ShellTable st, LutParam lp, Bands bd, int32_t N, int32_t npix, KeyOut o, Queues qs) {
  extern __shared__ __align__(128) uint8_t dyn[];
  float* ring = reinterpret_cast<float*>(dyn);                          // [kWStages][3 kWChunk]
  float4* lists = reinterpret_cast<float4*>(dyn + kWStages * kWChunk * 12);  // [warps][2][kWList]
  uint32_t* h32 = reinterpret_cast<uint32_t*>(dyn + kWSmemBase);          // 16-bit counters
  __shared__ FastShared fs;
  __shared__ __align__(8) uint64_t bar[kWStages];
  __shared__ int done_s[kWStages];
  __shared__ int abort_s;
  fast_init_shared(fs, bg, st, lp.v);
  const int nwords = (o.nbuckets + 1) >> 1;
  if (MODE == kModeDense && o.smem_hist)
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) h32[i] = 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kWStages; ++s) {
      mbar_init(&bar[s], 1);
      done_s[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_s = 0;
  }
  __syncthreads();

  const int lo = bg.shell_lo, hi = bg.shell_hi;
  const int n1 = 2 * bg.R + 1;
  const bool carry = bg.nimg == 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  float4* list_eq = lists + (2 * warp) * kWList;
  float4* list_cap = list_eq + kWList;
  const int64_t nchunks = (n + kWChunk - 1) / kWChunk;
  const int64_t mine = nchunks > blockIdx.x ? (nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t nfull = n / kWChunk;                   // chunks of kWChunk particles
  const int tail_n = int(n - nfull * kWChunk);         // particles of the last, partial chunk
  const int tail_smem = int(((uint32_t(tail_n) * 12u) & ~15u) / 12u);   // of them inside its copy
  auto chunk_bytes = [&](int64_t c) -> uint32_t {
    const int64_t rest = n - c * kWChunk;
    const int64_t cnt = rest < kWChunk ? rest : (int64_t)kWChunk;
    return uint32_t((cnt * 12) & ~15ll);       // bulk copies move multiples of 16 bytes
  };
  auto issue = [&](int64_t k) {                // k-th chunk of this block into stage k % kWStages
    const int64_t c = blockIdx.x + k * gridDim.x;
    const int s = int(k % kWStages);
    const uint32_t bytes = chunk_bytes(c);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], bytes);
    if (bytes) bulk_g2s(ring + s * 3 * kWChunk, xyz + c * kWChunk * 3, bytes, &bar[s]);
  };
  if (threadIdx.x == 0)
    for (int64_t kk = 0; kk < mine && kk < kWStages; ++kk) issue(kk);

  FastCtx fc{{-1, 0}, {-1, 0}, 0, 0};
  uint32_t* ghist = o.hist;
  int he = 0, ne = 0, hc = 0, nc = 0;          // heads and lengths of the two lists
  int ii = 0, jj = 0, kk = 0;                  // current image
  bool aborted = false;
  int64_t k = 0;
  // the shift of the only image when the box has no periodic images
  const float hsx = fs.shf[0][0], hsy = fs.shf[1][0], hsz = fs.shf[2][0];
  const float hlx = fs.shlo[0][0], hly = fs.shlo[1][0], hlz = fs.shlo[2][0];
  for (; k <= mine; ++k) {
    const bool last = k == mine;               // the final pass only drains the lists
    const int s = int(k & 1);                  // stage (two stages)
    if (!last) {
      if (!mbar_wait(&bar[s], uint32_t(k >> 1) & 1u)) {   // every lane waits (bounded)
        aborted = true;
        abort_s = 1;
      }
      if (__any_sync(0xFFFFFFFFu, aborted) || abort_s) { aborted = true; break; }
    }
    const int64_t kq = last ? (k > 0 ? k - 1 : 0) : k;   // chunk of the newest entries
    const int64_t cq = blockIdx.x + kq * gridDim.x;
    const int64_t base = cq * kWChunk;
    const bool fullc = cq < nfull;
    const int nvalid = last ? 0 : (fullc ? kWChunk : tail_n);
    const int nsmem = fullc ? kWChunk : tail_smem;      // particles inside the bulk copy
    const float* buf = ring + s * 3 * kWChunk;
    const uint32_t kqtag = uint32_t(kq & 4095) << 20;
    const int nimg = last ? 1 : bg.nimg;
    const bool drain_all = last || !carry || ((k & (kWAgeFlush - 1)) == kWAgeFlush - 1);
    const int ng = last ? 0 : kWGroups;                  // groups of 32 particles to classify
    const int nsteps = ng + (drain_all ? 1 : 0);         // + a drain step
    ii = jj = kk = 0;
#pragma unroll 1
    for (int img = 0; img < nimg; ++img) {
      if (img) {
        if (++kk == n1) { kk = 0; if (++jj == n1) { jj = 0; ++ii; } }
      }
      const float sx = IMAGES ? fs.shf[0][ii] : hsx, sy = IMAGES ? fs.shf[1][jj] : hsy,
                  sz = IMAGES ? fs.shf[2][kk] : hsz;
      const float lx = IMAGES ? fs.shlo[0][ii] : hlx, ly = IMAGES ? fs.shlo[1][jj] : hly,
                  lz = IMAGES ? fs.shlo[2][kk] : hlz;
      const uint64_t qbase = qpack(box_id, img, p_off + base);   // + offset in the chunk
#pragma unroll 1
      for (int h = 0; h < nsteps; ++h) {
        if (h < ng) {
          // ---- A: classify 32 particles of this warp's slice
          const int j = warp * kWPerWarp + 32 * h + lane;
          bool have;
          float x, y, zc;
          if (fullc) {                           // every particle inside the bulk copy
            have = true;
            x = buf[3 * j];
            y = buf[3 * j + 1];
            zc = buf[3 * j + 2];
          } else {
            have = j < nvalid;
            x = 0.f; y = 0.f; zc = 0.f;
            if (j < nsmem) {
              x = buf[3 * j];
              y = buf[3 * j + 1];
              zc = buf[3 * j + 2];
            } else if (have) {                   // ragged tail outside the bulk copy
              x = __ldg(xyz + 3 * (base + j));
              y = __ldg(xyz + 3 * (base + j) + 1);
              zc = __ldg(xyz + 3 * (base + j) + 2);
            }
          }
          const float dx = (x + sx) + lx;
          const float dy = (y + sy) + ly;
          const float dz = (zc + sz) + lz;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          // classification without branches but for the rare edge scan:
          // outside, undecided (c1), belt (c2) or cap (c3)
          const bool fin = r2 <= 3.0e38f;                // false for NaN and overflow
          const bool near = !(r2 >= bd.r2_min);          // near the observer (r == 0 is invalid)
          const float v = fminf(r2 * lp.scale, float(kLut - 1));
          const int bin = __float_as_int(v + 8388608.0f) - 0x4B000000;
          const uint32_t e = fs.lut[bin];
          int a = int(e & 0x7FFFu) - 1;
          bool band = false;
          // rare: scan the edges (finite r2 ends at +inf); a warp-uniform
          // test first, so that the common case is one vote and a branch
          if (__any_sync(0xFFFFFFFFu, (e & kLutScan) && fin)) {
            if ((e & kLutScan) && fin) {
              for (;;) {
                if (r2 < fs.lo2[a + 1]) break;
                if (r2 < fs.hi2[a + 1]) { band = true; break; }
                ++a;
              }
            }
          }
          const bool inshell = uint32_t(a - lo) < uint32_t(hi - lo);
          const float dz2 = dz * dz;
          const bool eqz = dz2 <= bd.z_eq2 * r2;
          const bool capz = dz2 > bd.z_cap2 * r2;
          const bool dec = have && fin && !near && !band && inshell;
          const bool c2 = dec && eqz;
          const bool c3 = dec && capz;
          // NaN or overflowing r2 (rare) goes to the queue as well, once per
          // particle (its first image): the FP64 stage returns the invalid
          // key for non-finite coordinates and decides a finite overflow
          const bool c1 = have && (fin ? (near || band || (inshell && !eqz && !capz))
                                       : (!IMAGES || img == 0));
          const uint32_t meta = uint32_t(a & 255) | (uint32_t(j) << 8) | kqtag;
          const float4 ent = make_float4(dx, dy, dz, __uint_as_float(meta));
          const unsigned meq = __ballot_sync(0xFFFFFFFFu, c2);
          const unsigned mcap = __ballot_sync(0xFFFFFFFFu, c3);
          if (c2) list_eq[(he + ne + __popc(meq & lt_mask)) & (kWList - 1)] = ent;
          if (c3) list_cap[(hc + nc + __popc(mcap & lt_mask)) & (kWList - 1)] = ent;
          ne += __popc(meq);
          nc += __popc(mcap);
          // undecided images wait in queue 1; outside/invalid are final
          bool pushed = true;                    // (a warp-uniform test first, as above)
          if (__any_sync(0xFFFFFFFFu, c1))
            pushed = queue_push(fc.qc, c1, qbase + uint64_t(j), qs.q1, qs.cap1, &qs.cnt->q1);
          if (!pushed) {
            const int32_t kx = key_exact_slow(st, lo, hi, N, npix, x, y, zc, bg.sh64[0][ii],
                                              bg.sh64[1][jj], bg.sh64[2][kk]);
            if (kx == kKeyInvalid) ++fc.n_invalid;
            if (kx >= 0) {
              ++fc.n_keyed;
              if (MODE == kModeDirect && UFC_IDX_OK(kx, o.ncell, 2)) atomicAdd(o.counts + kx, 1);
              if (MODE == kModeDense) {            // rare: straight to the global histogram
                const uint32_t dk = dense_key(kx, npix, o);
                if (UFC_IDX_OK(dk >> kOffBits, o.nbuckets, 1)) atomicAdd(ghist + (dk >> kOffBits), 1u);
                const unsigned long long at = atomicAdd(o.dense_count, 1ull);
                if ((int64_t)at < o.dense_cap) o.dense[at] = dk;
              }
            }
            if (MODE == kModeKeys && have) o.keys[p_off + base + j] = kx;
          } else if (MODE == kModeKeys && have && !c2 && !c3) {
            o.keys[p_off + base + j] = c1 ? kKeyUndecided
                : ((!fin && !(isfinite(x) && isfinite(y) && isfinite(zc))) ? kKeyInvalid : kKeyOutside);
          }
        }
        __syncwarp();
        // ---- B: pixels of full groups of 32 pending entries (in the drain
        // step, also of the partial rest)
        const bool tail = h == ng;
        // one instantiation per zone, so that a group runs only its zone's
        // pixel code
        auto group_b = [&](auto zone_tag, int take) {
          constexpr int ZONE = decltype(zone_tag)::value;
          const float4* L = ZONE == 0 ? list_eq : list_cap;
          const int head = ZONE == 0 ? he : hc;
          const bool have = lane < take;
          float4 ent = make_float4(0.f, 0.f, 0.f, 0.f);
          if (have) ent = L[(head + lane) & (kWList - 1)];
          if constexpr (ZONE == 0) { he = (he + take) & (kWList - 1); ne -= take; }
          else { hc = (hc + take) & (kWList - 1); nc -= take; }
          const float dx = ent.x, dy = ent.y, dz = ent.z;
          const uint32_t meta = __float_as_uint(ent.w);
          const int b = int(meta & 255u);
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const float rinv = rsqrtf(r2);
          const float z = dz * rinv;
          int32_t pix = kKeyUndecided;
          if (have) {
            if constexpr (ZONE == 0) pix = pixel_fast_eq(N, bd, dx, dy, z);
            else pix = pixel_fast_cap(N, bd, dx, dy, dz, r2, rinv, z);
          }
          const bool ok = have && pix != kKeyUndecided;
          // the entry's particle (launch-local index pl): chunk from the
          // 12-bit tag, offset in the chunk; computed only where needed
          auto local_index = [&]() -> int64_t {
            const int64_t ke = kq - ((kq - int64_t(meta >> 20)) & 4095);
            return (blockIdx.x + ke * gridDim.x) * kWChunk + int64_t((meta >> 8) & 4095u);
          };
          const int32_t key = b * npix + pix;
          bool queued = true;
          if (__any_sync(0xFFFFFFFFu, have && !ok)) {   // rare: a warp-uniform test first
            if constexpr (IMAGES) {
              queued = queue_push_f(
                  fc.qc, have && !ok, [&]() { return qpack(box_id, img, p_off + local_index()); },
                  qs.q1, qs.cap1, &qs.cnt->q1);
            } else {                             // queue full: left to the exact pass
              queue_push_mark(
                  fc.qc, have && !ok, [&]() { return qpack(box_id, 0, p_off + local_index()); },
                  qs.q1, qs.cap1, &qs.cnt->q1, qs.ovf, qs.ovf_base, &qs.cnt->ovf);
            }
          }
          if (!queued) {                         // queue full: the FP64 procedure here
            const int64_t pl = local_index();
            const float x = __ldg(xyz + 3 * pl), y = __ldg(xyz + 3 * pl + 1),
                        zc = __ldg(xyz + 3 * pl + 2);
            const int32_t kx = key_exact_slow(st, lo, hi, N, npix, x, y, zc, bg.sh64[0][ii],
                                              bg.sh64[1][jj], bg.sh64[2][kk]);
            if (kx >= 0) {
              ++fc.n_keyed;
              if (MODE == kModeDirect && UFC_IDX_OK(kx, o.ncell, 2)) atomicAdd(o.counts + kx, 1);
              if (MODE == kModeDense) {
                const uint32_t dk = dense_key(kx, npix, o);
                if (UFC_IDX_OK(dk >> kOffBits, o.nbuckets, 1)) atomicAdd(ghist + (dk >> kOffBits), 1u);
                const unsigned long long at = atomicAdd(o.dense_count, 1ull);
                if ((int64_t)at < o.dense_cap) o.dense[at] = dk;
              }
            }
            if (MODE == kModeKeys) o.keys[p_off + pl] = kx;
          }
          if (MODE == kModeKeys) {
            if (have && queued) o.keys[p_off + local_index()] = ok ? key : kKeyUndecided;
          } else if (MODE == kModeDirect) {
            if (ok && UFC_IDX_OK(key, o.ncell, 2)) atomicAdd(o.counts + key, 1);
          } else {
            uint32_t dk = 0u, bucket = 0u;
            bool wrapped = false;
            if (ok) {
              const uint32_t blk = uint32_t(pix >> 13) / 3u;       // pix / 24576
              bucket = uint32_t(b - o.shell0) * uint32_t(o.nblk) + blk;
              dk = (bucket << kOffBits) | (uint32_t(pix) - blk * uint32_t(kBlockPix));
              if (UFC_IDX_OK(bucket, o.nbuckets, 1)) {
                if (o.smem_hist) wrapped = hist16_add(h32, bucket);
                else atomicAdd(ghist + bucket, 1u);
              }
            }
            // rare (one increment in 65536 per counter): a warp-uniform test first
            if (__any_sync(0xFFFFFFFFu, wrapped) && wrapped) hist16_carry(h32, ghist, bucket);
            dense_append(fc.wc, ok, dk, o);
          }
          fc.n_keyed += ok;
        };
        const int take_e = ne >= 32 ? 32 : ((tail && drain_all) ? ne : 0);
        if (take_e) group_b(std::integral_constant<int, 0>{}, take_e);
        const int take_c = nc >= 32 ? 32 : ((tail && drain_all) ? nc : 0);
        if (take_c) group_b(std::integral_constant<int, 1>{}, take_c);
        __syncwarp();
      }
    }
    if (last) break;
    // this warp is done with stage s; the last warp refills it
    if (lane == 0) {
      __threadfence_block();
      const int prev = atomicAdd(&done_s[s], 1);
      if (prev == kWWarps - 1) {
        atomicExch(&done_s[s], 0);
        if (k + kWStages < mine) issue(k + kWStages);
      }
    }
    __syncwarp();
  }
  if (aborted) {
    // a wait ran out: report, then wait (bounded) for the copies that may
    // still be in flight into this block's shared memory, and leave
    if (lane == 0) {
      atomicAdd(&qs.cnt->timeouts, 1ull);
      for (int64_t q = k; q < mine && q < k + kWStages; ++q)
        mbar_wait(&bar[q % kWStages], uint32_t((q / kWStages) & 1));
    }
    return;
  }
  // ---- end: close the warp's chunks, counters, bucket counts
  if (MODE == kModeDense) dense_close(fc.wc, o);
  queue_close(fc.qc, qs.q1, qs.cap1);
  const unsigned long long ni = warp_sum(fc.n_invalid), nk = warp_sum(fc.n_keyed);
  if (lane == 0) {
    if (ni) atomicAdd(&qs.cnt->invalid, ni);
    if (nk) atomicAdd(&qs.cnt->keyed, nk);
  }
  if (MODE == kModeDense && o.smem_hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < o.nbuckets; i += blockDim.x) {
      const uint32_t v = (h32[i >> 1] >> ((i & 1) << 4)) & 0xFFFFu;
      if (v) atomicAdd(ghist + i, v);
    }
  }
}

// ------------------------------------------------ refine and exact stages --
template <int MODE>
__device__ __forceinline__ void emit_late(int32_t key, int64_t p, int32_t npix,
                                          const KeyOut& o, WarpChunk& wc) {
  if (MODE == kModeKeys) {
    o.keys[p] = key;
  } else if (MODE == kModeDirect) {
    if (key >= 0 && UFC_IDX_OK(key, o.ncell, 2)) atomicAdd(o.counts + key, 1);
  } else {
    uint32_t dk = key >= 0 ? dense_key(key, npix, o) : 0u;
    if (key >= 0 && UFC_IDX_OK(dk >> kOffBits, o.nbuckets, 1)) atomicAdd(o.hist + (dk >> kOffBits), 1u);
    dense_append(wc, key >= 0, dk, o);
  }
}

struct BoxesParam {
  BoxGeom box[kMaxBoxes];
  const float* xyz[kMaxBoxes];
  int64_t n[kMaxBoxes];          // particles of each box in this call
  int64_t bit_base[kMaxBoxes];   // first overflow bit of each box (boxes without images)
};

template <int MODE>
__global__ void __launch_bounds__(256)
k_refine(BoxesParam bp, ShellTable st, int32_t N, int32_t npix, KeyOut o, Queues qs) {
  __shared__ float chih_s[kMaxShells + 1], chil_s[kMaxShells + 1];
  __shared__ float2 atab_s[kAtanTab];
  for (int i = threadIdx.x; i <= st.nshell; i += blockDim.x) {
    chih_s[i] = st.chih[i];
    chil_s[i] = st.chil[i];
  }
  fill_atan_table(atab_s);
  __syncthreads();
  const unsigned long long total = qs.cnt->q1;
  const int64_t m = (int64_t)min((unsigned long long)qs.cap1, total);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (m + stride - 1) / stride;
  WarpChunk wc{-1, 0};
  unsigned long long n_ref = 0, n_invalid = 0, n_keyed = 0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  QChunk qc{-1, 0};
  for (int64_t it = 0; it < iters; ++it, i += stride) {
    bool have = i < m;
    int32_t key = kKeyOutside;
    int64_t p = 0;
    uint64_t e = 0;
    if (have) e = qs.q1[i];
    have = have && e != kQEmpty;
    if (have) {
      const int b = qbox(e), img = qimg(e);
      p = qidx(e);
      const BoxGeom& g = bp.box[b];
      int ii = 0, jj = 0, kk = 0;
      if (g.R) {                                   // periodic images only
        const int n1 = 2 * g.R + 1;
        ii = img / (n1 * n1); jj = (img / n1) % n1; kk = img % n1;
      }
      const float* xp = bp.xyz[b] + 3 * p;
      float x = xp[0], y = xp[1], zc = xp[2];
      key = key_refine(chih_s, chil_s, atab_s, g.shell_lo, g.shell_hi, N, npix, x, y, zc, g.shf[0][ii],
                       g.shf[1][jj], g.shf[2][kk], g.shlo[0][ii], g.shlo[1][jj],
                       g.shlo[2][kk]);
      ++n_ref;
    }
    const bool und = have && key == kKeyUndecided;
    if (!queue_push(qc, und, e, qs.q2, qs.cap2, &qs.cnt->q2)) {
      const int b = qbox(e), img = qimg(e);
      const BoxGeom& g = bp.box[b];
      const int n1 = 2 * g.R + 1;
      const int ii = img / (n1 * n1), jj = (img / n1) % n1, kk = img % n1;
      const float* xp = bp.xyz[b] + 3 * p;
      key = key_exact(st, g.shell_lo, g.shell_hi, N, npix, xp[0], xp[1], xp[2],
                      g.sh64[0][ii], g.sh64[1][jj], g.sh64[2][kk]);
      if (key == kKeyInvalid) ++n_invalid;
    }
    const bool done = have && key != kKeyUndecided;
    n_keyed += done && key >= 0;
    if (MODE == kModeDense) {
      emit_late<MODE>(done ? key : kKeyOutside, p, npix, o, wc);
    } else if (done) {
      emit_late<MODE>(key, p, npix, o, wc);
    }
  }
  if (MODE == kModeDense) dense_close(wc, o);
  queue_close(qc, qs.q2, qs.cap2);
  n_ref = warp_sum(n_ref);
  n_invalid = warp_sum(n_invalid);
  n_keyed = warp_sum(n_keyed);
  if ((threadIdx.x & 31) == 0) {
    if (n_ref) atomicAdd(&qs.cnt->refined, n_ref);
    if (n_invalid) atomicAdd(&qs.cnt->invalid, n_invalid);
    if (n_keyed) atomicAdd(&qs.cnt->keyed, n_keyed);
  }
}

template <int MODE>
__global__ void __launch_bounds__(256)
k_exact(BoxesParam bp, ShellTable st, int32_t N, int32_t npix, KeyOut o, Queues qs) {
  const unsigned long long total = qs.cnt->q2;
  const int64_t m = (int64_t)min((unsigned long long)qs.cap2, total);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (m + stride - 1) / stride;
  WarpChunk wc{-1, 0};
  unsigned long long n_ex = 0, n_invalid = 0, n_keyed = 0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < iters; ++it, i += stride) {
    bool have = i < m;
    int32_t key = kKeyOutside;
    int64_t p = 0;
    uint64_t e = kQEmpty;
    if (have) e = qs.q2[i];
    have = have && e != kQEmpty;
    if (have) {
      const int b = qbox(e), img = qimg(e);
      p = qidx(e);
      const BoxGeom& g = bp.box[b];
      const int n1 = 2 * g.R + 1;
      const int ii = img / (n1 * n1), jj = (img / n1) % n1, kk = img % n1;
      const float* xp = bp.xyz[b] + 3 * p;
      key = key_exact(st, g.shell_lo, g.shell_hi, N, npix, xp[0], xp[1], xp[2],
                      g.sh64[0][ii], g.sh64[1][jj], g.sh64[2][kk]);
      ++n_ex;
      if (key == kKeyInvalid) ++n_invalid;
      n_keyed += key >= 0;
    }
    if (MODE == kModeDense) emit_late<MODE>(have ? key : kKeyOutside, p, npix, o, wc);
    else if (have) emit_late<MODE>(key, p, npix, o, wc);
  }
  if (MODE == kModeDense) dense_close(wc, o);
  n_ex = warp_sum(n_ex);
  n_invalid = warp_sum(n_invalid);
  n_keyed = warp_sum(n_keyed);
  if ((threadIdx.x & 31) == 0) {
    if (n_ex) atomicAdd(&qs.cnt->exact, n_ex);
    if (n_invalid) atomicAdd(&qs.cnt->invalid, n_invalid);
    if (n_keyed) atomicAdd(&qs.cnt->keyed, n_keyed);
  }
}

// Exact pass over the images the fast stage could neither decide nor queue
// (queue 1 full; boxes without periodic images): one bit per particle of
// those boxes.  Returns at once unless the fast stage marked any.
template <int MODE>
__global__ void __launch_bounds__(256)
k_overflow(BoxesParam bp, int nbox, ShellTable st, int32_t N, int32_t npix, KeyOut o, Queues qs,
           int64_t nwords) {
  if (qs.cnt->ovf == 0ull) return;
  unsigned long long n_ex = 0, n_invalid = 0, n_keyed = 0;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t m = qs.ovf[w];
    while (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1u;
      const int64_t idx = w * 32 + bit;
      int k = 0;
      while (k + 1 < nbox && bp.bit_base[k + 1] <= idx) ++k;
      const int64_t p = idx - bp.bit_base[k];
      const BoxGeom& g = bp.box[k];
      const float* xp = bp.xyz[k] + 3 * p;
      const int32_t key = key_exact(st, g.shell_lo, g.shell_hi, N, npix, xp[0], xp[1], xp[2],
                                    g.sh64[0][0], g.sh64[1][0], g.sh64[2][0]);
      ++n_ex;
      if (key == kKeyInvalid) ++n_invalid;
      if (MODE == kModeKeys) o.keys[p] = key;
      if (key >= 0) {
        ++n_keyed;
        if (MODE == kModeDirect && UFC_IDX_OK(key, o.ncell, 2)) atomicAdd(o.counts + key, 1);
        if (MODE == kModeDense) {
          const uint32_t dk = dense_key(key, npix, o);
          if (UFC_IDX_OK(dk >> kOffBits, o.nbuckets, 1)) atomicAdd(o.hist + (dk >> kOffBits), 1u);
          const unsigned long long at = atomicAdd(o.dense_count, 1ull);
          if ((int64_t)at < o.dense_cap) o.dense[at] = dk;
        }
      }
    }
  }
  if (n_ex) atomicAdd(&qs.cnt->exact, n_ex);
  if (n_invalid) atomicAdd(&qs.cnt->invalid, n_invalid);
  if (n_keyed) atomicAdd(&qs.cnt->keyed, n_keyed);
}

// ------------------------------------------------------ dense pipeline -----
// Exclusive scan of hist[nb] into off[nb+1] (one block of 1024 threads).
__global__ void __launch_bounds__(1024) k_scan(const uint32_t* __restrict__ hist, int nb,
                                               int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int a = t * per, b = min(nb, a + per);
  int64_t s = 0;
  for (int i = a; i < b; ++i) s += hist[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = t ? part[t - 1] : 0;
  for (int i = a; i < b; ++i) {
    off[i] = run;
    run += hist[i];
  }
  if (t == 1023) off[nb] = part[1023];
}

// Cursor initialisation: gcur[g] = off[g << kGroupBits], bcur[b] = off[b].
__global__ void k_cursors(const int64_t* __restrict__ off, int nb, int ng,
                          unsigned long long* __restrict__ gcur,
                          unsigned long long* __restrict__ bcur) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) bcur[i] = (unsigned long long)off[i];
  if (i < ng) gcur[i] = (unsigned long long)off[min(nb, i << kGroupBits)];
}

// Exclusive scan of cnt[0..n) into start[] by the first warp.
__device__ __forceinline__ void warp_exclusive_scan(const uint32_t* cnt, uint32_t* start, int n) {
  const int lane = threadIdx.x & 31;
  const int per = (n + 31) / 32;
  const int a = lane * per, b = min(n, a + per);
  uint32_t s = 0;
  for (int i = a; i < b; ++i) s += cnt[i];
  uint32_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  uint32_t run = incl - s;
  for (int i = a; i < b; ++i) { start[i] = run; run += cnt[i]; }
}

constexpr int kScatThreads = 512;
constexpr int kScatPer = 16;
constexpr int kScatTile = kScatThreads * kScatPer;   // 8192 keys: ~64 B per destination

// Two-buffer prefetch of scatter tiles: while a block works on one tile, the
// bulk copy of its tile after next streams into the other buffer (tracked by
// mbarriers with bounded waits).  A copy moves whole 16-byte units from a
// 16-byte aligned address; the ragged end of a tile comes from plain loads.
struct TilePrefetch {
  uint64_t* bar;        // [2]
  uint32_t* buf;        // [2][kScatTile + 4]
  __device__ void init() {
    if (threadIdx.x == 0) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  // keys [a0, a0 + nkeys) of src (a0 a multiple of 4) into buffer b
  __device__ void issue(int b, const uint32_t* src, int64_t a0, int nkeys) {
    const uint32_t bytes = uint32_t(nkeys * 4) & ~15u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[b], bytes);
    if (bytes) bulk_g2s(buf + b * (kScatTile + 4), src + a0, bytes, &bar[b]);
  }
  __device__ bool wait(int b, int64_t use) { return mbar_wait(&bar[b], uint32_t(use & 1)); }
};

// Pass A: dense keys -> grouped array, group = bucket >> kGroupBits.  Two
// blocks per SM: one block's prefetch and global atomics overlap the other's
// counting, scan and write-out phases.  Each destination's offset is kept as
// (global base - tile start), one 64-bit shared load per key at write-out.
__global__ void __launch_bounds__(kScatThreads, 2)
k_scatter_group(const uint32_t* __restrict__ dense, const unsigned long long* dense_count,
                int64_t dense_cap, int ng, unsigned long long* __restrict__ gcur,
                uint32_t* __restrict__ out, unsigned long long* timeouts) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ __align__(8) uint64_t bar[2];
  TilePrefetch pf{bar, sm};                // [2][kScatTile + 4]
  uint32_t* tile = sm + 2 * (kScatTile + 4);                       // [kScatTile]
  unsigned long long* base = (unsigned long long*)(tile + kScatTile);  // [ng], 8-aligned
  uint32_t* cnt = (uint32_t*)(base + ng);  // [ng]
  uint32_t* start = cnt + ng;              // [ng]
  const int64_t total = (int64_t)min(*dense_count, (unsigned long long)dense_cap);
  const int64_t ntiles = (total + kScatTile - 1) / kScatTile;
  const int64_t mine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int shift = kOffBits + kGroupBits;
  auto tile_keys = [&](int64_t i) -> int {   // keys of this block's i-th tile
    const int64_t t0 = (blockIdx.x + i * gridDim.x) * (int64_t)kScatTile;
    return int(min((int64_t)kScatTile, total - t0));
  };
  pf.init();
  __syncthreads();
  if (threadIdx.x == 0)
    for (int64_t i = 0; i < mine && i < 2; ++i)
      pf.issue(int(i), dense, (blockIdx.x + i * gridDim.x) * (int64_t)kScatTile, tile_keys(i));
  uint32_t v[kScatPer];
  int64_t i = 0;
  bool aborted = false;
  for (; i < mine; ++i) {
    const int b = int(i & 1);
    const int64_t t0 = (blockIdx.x + i * gridDim.x) * (int64_t)kScatTile;
    const int nk = tile_keys(i);
    const int nsm = (nk * 4 & ~15) / 4;      // keys inside the bulk copy
    const bool ok = pf.wait(b, i >> 1);
    const uint32_t* kb = pf.buf + b * (kScatTile + 4);
#pragma unroll
    for (int k = 0; k < kScatPer; ++k) {
      const int j = k * kScatThreads + threadIdx.x;
      v[k] = j < nsm ? kb[j] : (j < nk ? __ldcs(dense + t0 + j) : kSentinel);
      if (v[k] != kSentinel && !UFC_IDX_OK(v[k] >> shift, ng, 3)) v[k] = kSentinel;
    }
    for (int g = threadIdx.x; g < ng; g += blockDim.x) cnt[g] = 0;
    if (__syncthreads_or(!ok)) { aborted = true; break; }   // buffer b is free again
    if (threadIdx.x == 0 && i + 2 < mine)
      pf.issue(b, dense, t0 + 2ll * gridDim.x * kScatTile, tile_keys(i + 2));
    uint32_t slot[kScatPer];
#pragma unroll
    for (int k = 0; k < kScatPer; ++k)
      slot[k] = v[k] != kSentinel ? atomicAdd(cnt + (v[k] >> shift), 1u) : 0u;
    __syncthreads();
    if (threadIdx.x < 32) warp_exclusive_scan(cnt, start, ng);
    __syncthreads();
    for (int g = threadIdx.x; g < ng; g += blockDim.x)
      base[g] = (cnt[g] ? atomicAdd(gcur + g, (unsigned long long)cnt[g]) : 0ull) - start[g];
#pragma unroll
    for (int k = 0; k < kScatPer; ++k)
      if (v[k] != kSentinel) tile[start[v[k] >> shift] + slot[k]] = v[k];
    __syncthreads();
    const uint32_t used = start[ng - 1] + cnt[ng - 1];
    for (uint32_t q = threadIdx.x; q < used; q += blockDim.x) {
      const uint32_t val = tile[q];
      const uint32_t g = val >> shift;
      if (UFC_IDX_OK(base[g] + q, dense_cap, 4)) out[base[g] + q] = val;
    }
    __syncthreads();
  }
  if (aborted && threadIdx.x == 0) {         // report; wait (bounded) for copies in flight
    atomicAdd(timeouts, 1ull);
    for (int64_t q = i; q < mine && q < i + 2; ++q) pf.wait(int(q & 1), q >> 1);
  }
}

struct Tile { int32_t group; int32_t len; int64_t start; };

// Tile list of pass B: every group's range split into kScatTile pieces.
// Every block scans the per-group tile counts in shared memory (ng + 1
// entries), then the grid writes the tiles, each thread finding its tile's
// group by binary search over the scan.
constexpr int kTilesThreads = 256;
__global__ void __launch_bounds__(kTilesThreads) k_tiles(const int64_t* __restrict__ off, int nb,
                                                         int ng, Tile* __restrict__ tiles,
                                                         unsigned long long* __restrict__ ntiles) {
  extern __shared__ int64_t tsm[];
  int64_t* gs = tsm;                 // [ng + 1] first key of each group, then the end
  int64_t* pre = tsm + ng + 1;       // [ng + 1] first tile of each group, then the total
  for (int g = threadIdx.x; g <= ng; g += blockDim.x) gs[g] = off[min(nb, g << kGroupBits)];
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int g = 0; g < ng; ++g) {
      pre[g] = run;
      run += (gs[g + 1] - gs[g] + kScatTile - 1) / kScatTile;
    }
    pre[ng] = run;
  }
  __syncthreads();
  const int64_t total = pre[ng];
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total;
       w += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = ng;                           // pre[lo] <= w < pre[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= w) lo = mid; else hi = mid;
    }
    const int64_t st = gs[lo] + (w - pre[lo]) * kScatTile;
    const int64_t len = gs[lo + 1] - st;
    tiles[w] = Tile{lo, (int32_t)(len < kScatTile ? len : kScatTile), st};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *ntiles = (unsigned long long)total;
}

// Pass B: grouped keys -> per-bucket u16 offsets (two blocks per SM and the
// same tile prefetch as pass A; a tile starts anywhere, so its copy starts
// at the 16-byte unit holding its first key, and the grouped array has 4
// keys of slack at its end).  The tile keeps each whole key, so that one
// 32-bit shared store per key places it and the write-out reads the
// destination digit back from the key.
__global__ void __launch_bounds__(kScatThreads, 2)
k_scatter_bucket(const uint32_t* __restrict__ grouped, const Tile* __restrict__ tiles,
                 const unsigned long long* __restrict__ ntiles_p,
                 unsigned long long* __restrict__ bcur, uint16_t* __restrict__ out,
                 int64_t out_cap, unsigned long long* timeouts) {
  constexpr int NS = 1 << kGroupBits;
  extern __shared__ __align__(16) uint8_t smb[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ Tile tb[2];
  TilePrefetch pf{bar, reinterpret_cast<uint32_t*>(smb)};                  // [2][kScatTile + 4]
  unsigned long long* base =
      reinterpret_cast<unsigned long long*>(smb + 2 * (kScatTile + 4) * 4);  // [NS]
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + NS);                  // [NS]
  uint32_t* start = cnt + NS;                                              // [NS]
  uint32_t* tile = start + NS;                                             // [kScatTile]
  const int64_t ntiles = (int64_t)*ntiles_p;
  const int64_t mine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto tile_at = [&](int64_t i) -> const Tile& { return tiles[blockIdx.x + i * gridDim.x]; };
  auto issue = [&](int b, const Tile& t) {   // thread 0
    tb[b] = t;
    const int64_t a0 = t.start & ~3ll;
    pf.issue(b, grouped, a0, int(t.start - a0) + t.len + 3);   // whole units up to the end
  };
  pf.init();
  __syncthreads();
  Tile nxt{0, 0, 0};                          // thread 0: the tile after next
  if (threadIdx.x == 0) {
    for (int64_t i = 0; i < mine && i < 2; ++i) issue(int(i), tile_at(i));
    if (mine > 2) nxt = tile_at(2);
  }
  __syncthreads();
  uint32_t v[kScatPer];
  int64_t i = 0;
  bool aborted = false;
  for (; i < mine; ++i) {
    const int b = int(i & 1);
    const Tile T = tb[b];
    const int64_t a0 = T.start & ~3ll;
    const bool ok = pf.wait(b, i >> 1);
    const uint32_t* kb = pf.buf + b * (kScatTile + 4) + (T.start - a0);   // the copy holds every key
#pragma unroll
    for (int k = 0; k < kScatPer; ++k) {
      const int j = k * kScatThreads + threadIdx.x;
      v[k] = j < T.len ? kb[j] : kSentinel;
    }
    for (int q = threadIdx.x; q < NS; q += blockDim.x) cnt[q] = 0;
    if (__syncthreads_or(!ok)) { aborted = true; break; }   // buffer b and tb[b] are free
    if (threadIdx.x == 0 && i + 2 < mine) {
      issue(b, nxt);
      if (i + 3 < mine) nxt = tile_at(i + 3);
    }
    uint32_t slot[kScatPer];
#pragma unroll
    for (int k = 0; k < kScatPer; ++k)
      slot[k] = v[k] != kSentinel ? atomicAdd(cnt + ((v[k] >> kOffBits) & (NS - 1)), 1u) : 0u;
    __syncthreads();
    if (threadIdx.x < 32) warp_exclusive_scan(cnt, start, NS);
    __syncthreads();
    for (int sIdx = threadIdx.x; sIdx < NS; sIdx += blockDim.x)
      base[sIdx] = (cnt[sIdx] ? atomicAdd(bcur + ((int64_t)T.group << kGroupBits) + sIdx,
                                          (unsigned long long)cnt[sIdx]) : 0ull) - start[sIdx];
#pragma unroll
    for (int k = 0; k < kScatPer; ++k)
      if (v[k] != kSentinel) {
        const uint32_t sub = (v[k] >> kOffBits) & (NS - 1);
        tile[start[sub] + slot[k]] = v[k];
      }
    __syncthreads();
    for (int q = threadIdx.x; q < T.len; q += blockDim.x) {
      const uint32_t val = tile[q];
      const unsigned long long dst = base[(val >> kOffBits) & (NS - 1)] + q;
      if (UFC_IDX_OK(dst, out_cap, 5)) out[dst] = uint16_t(val & ((1u << kOffBits) - 1u));
    }
    __syncthreads();
  }
  if (aborted && threadIdx.x == 0) {         // report; wait (bounded) for copies in flight
    atomicAdd(timeouts, 1ull);
    for (int64_t q = i; q < mine && q < i + 2; ++q) pf.wait(int(q & 1), q >> 1);
  }
}

// Count map of each bucket from its u16 offsets, in shared memory.  The
// bucket's offsets are read with 16-byte loads (8 offsets each), up to
// kHistVec per thread in flight, plus scalar head and tail.  The write-out
// of a bucket also clears its shared counters for the next one.  When
// accumulating, a bucket without particles leaves its block of the map
// untouched.
constexpr int kHistThreads = 512;
constexpr int kHistVec = 8;
__global__ void __launch_bounds__(kHistThreads)
k_hist_block(const uint16_t* __restrict__ offs, const int64_t* __restrict__ off, int nb,
             int32_t* __restrict__ counts, int accumulate, int64_t offs_cap) {
  extern __shared__ uint32_t h[];   // [kBlockPix]
  uint4* h4 = reinterpret_cast<uint4*>(h);
  for (int i = threadIdx.x; i < kBlockPix / 4; i += blockDim.x) h4[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t a = off[b];
    int64_t e = off[b + 1];
    if (e > a && !UFC_IDX_OK(e - 1, offs_cap, 6)) e = a;   // (checked) a bucket beyond the array
    if (accumulate && a == e) continue;          // nothing to add (uniform over the block)
    const int64_t a8r = (a + 7) & ~7ll, e8r = e & ~7ll;
    const int64_t a8 = a8r < e ? a8r : e;                  // first 16-byte boundary
    const int64_t e8 = e8r > a8 ? e8r : a8;                // last one
    if (threadIdx.x < a8 - a) {
      const uint32_t v = offs[a + threadIdx.x];
      if (UFC_IDX_OK(v, kBlockPix, 7)) atomicAdd(h + v, 1u);
    }
    if (threadIdx.x < e - e8) {
      const uint32_t v = offs[e8 + threadIdx.x];
      if (UFC_IDX_OK(v, kBlockPix, 7)) atomicAdd(h + v, 1u);
    }
    const uint4* body = reinterpret_cast<const uint4*>(offs + a8);
    const int64_t nvec = (e8 - a8) >> 3;
    for (int64_t i0 = threadIdx.x; i0 < nvec; i0 += kHistVec * kHistThreads) {
      uint4 q[kHistVec];
#pragma unroll
      for (int k = 0; k < kHistVec; ++k) {
        const int64_t i = i0 + k * kHistThreads;
        q[k] = i < nvec ? __ldcs(body + i) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < kHistVec; ++k) {
        if (i0 + k * kHistThreads < nvec) {
          const uint32_t w[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (UFC_IDX_OK(w[j] & 0xFFFFu, kBlockPix, 7)) atomicAdd(h + (w[j] & 0xFFFFu), 1u);
            if (UFC_IDX_OK(w[j] >> 16, kBlockPix, 7)) atomicAdd(h + (w[j] >> 16), 1u);
          }
        }
      }
    }
    __syncthreads();
    int4* dst = reinterpret_cast<int4*>(counts + (int64_t)b * kBlockPix);
    for (int i = threadIdx.x; i < kBlockPix / 4; i += blockDim.x) {
      const uint4 sv = h4[i];
      h4[i] = make_uint4(0, 0, 0, 0);
      int4 d = make_int4(int(sv.x), int(sv.y), int(sv.z), int(sv.w));
      if (accumulate) {
        const int4 o = dst[i];
        d.x += o.x; d.y += o.y; d.z += o.z; d.w += o.w;
      }
      __stcs(dst + i, d);
    }
    __syncthreads();
  }
}

// ================================================================ host ======

// Index-check record of this translation unit (checked builds), read and
// cleared on the context stream.
cudaError_t take_checks_bin(CheckRec* out, cudaStream_t s) { return take_check_rec(out, s); }

// A failed index test on purpose (every build): index i against bound n at
// site 0.  The test records and skips; nothing is accessed.
__global__ void k_check_selftest(long long i, long long n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) check_idx(i, n, 0);
}
ufc_status run_check_selftest(ufc_ctx* c, int64_t index, int64_t bound) {
  k_check_selftest<<<1, 32, 0, c->stream>>>((long long)index, (long long)bound);
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

static float f_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = nextafterf(f, -INFINITY);
  return f;
}
static float f_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = nextafterf(f, INFINITY);
  return f;
}

// FP32-stage bands (error analysis in pixel.cuh and DESIGN):
//  r2  : |r2f - R2| <= 7u R2      -> band 14u (x2)
//  z   : |zf - Z| <= 10.5u |Z|   -> band 21u
//  eq  : |w - W| <= 14u N (+u)   -> band 28u N + 2u
//  cap : |v - V| <= 29u N        -> band 58u N + 2u
//  ip  : |w3 - W3| <= 7.5u ir    -> band 15u ir (+2u)
// plus guards that keep the absolute input error (2u^2 smax) negligible.
// The eq and cap fields hold 1/2 - band - 2^-23 (rounded down); eq_d and
// cap_d are 1/2 minus them (at least band + 2^-23), the least distance from
// the nearest integer that the fast stage's floor test accepts.
static void make_bands(int N, float smax, Bands& bd) {
  const double u = std::ldexp(1.0, -24);
  bd.fN = (float)N;
  bd.n75 = 0.75f * (float)N;
  bd.c0 = N == 1 ? 0.5f : 0.0f;
  bd.nhalf = N >> 1;
  bd.ring0 = 2 * N * (N - 1);
  bd.four_n = 4 * N;
  bd.eight_n = 8 * N;
  bd.npix = 12 * N * N;
  const double two3 = 2.0 / 3.0;
  bd.z_eq = f_down(two3 / (1.0 + 21.0 * u) * (1.0 - 1e-12));
  bd.z_cap = f_up(two3 / (1.0 - 21.0 * u) * (1.0 + 1e-12));
  bd.eq = f_down(0.5 - f_up(28.0 * u * N + 2.0 * u) - std::ldexp(1.0, -23));
  bd.cap = f_down(0.5 - f_up(58.0 * u * N + 2.0 * u) - std::ldexp(1.0, -23));
  bd.eq_d = 0.5f - bd.eq;     // exact (Sterbenz)
  bd.cap_d = 0.5f - bd.cap;
  bd.ip_per_ir = f_up(17.0 * u);
  double g = std::ldexp(1.0, 11) * u * std::max<double>(smax, 1.0);
  bd.r2_min = f_up(g * g);
  bd.axy_min = f_up(g);
  // zone by squares: dz^2 (<= 5u), r2 (<= 6u) and z2 r2 (u) give z^2 within
  // 12u relative of the exact value above r2_min; the band is twice that
  bd.z_eq2 = f_down(4.0 / 9.0 / (1.0 + 24.0 * u) * (1.0 - 1e-12));
  bd.z_cap2 = f_up(4.0 / 9.0 / (1.0 - 24.0 * u) * (1.0 + 1e-12));
}

static ufc_status make_table(ufc_ctx* c, const double* chi, int nshell, ShellTable& st) {
  const double u = std::ldexp(1.0, -24);
  std::memset(&st, 0, sizeof st);
  st.nshell = nshell;
  for (int e = 0; e <= nshell; ++e) {
    if (!std::isfinite(chi[e]) || chi[e] < 0.0)
      return set_err(c, UFC_ERR_ARG, "chi_edges[%d] = %g is not a finite radius >= 0", e, chi[e]);
    if (e > 0 && !(chi[e] > chi[e - 1]))
      return set_err(c, UFC_ERR_ARG, "chi_edges must increase (edge %d)", e);
    st.chi64[e] = chi[e];
    st.chih[e] = (float)chi[e];
    st.chil[e] = (float)(chi[e] - (double)st.chih[e]);
    double c2 = chi[e] * chi[e];
    st.lo2[e] = f_down(c2 * (1.0 - 14.0 * u) * (1.0 - 1e-12));
    st.hi2[e] = f_up(c2 * (1.0 + 14.0 * u) * (1.0 + 1e-12));
    if (e > 0 && !(st.hi2[e - 1] <= st.lo2[e]))
      return set_err(c, UFC_ERR_UNSUPPORTED,
                     "shell edges %d and %d are closer than 3e-6 relative", e - 1, e);
  }
  return UFC_OK;
}

static ufc_status make_box(ufc_ctx* c, const ufc_box& b, int nshell, BoxGeom& g) {
  std::memset(&g, 0, sizeof g);
  if (!(b.L > 0.0) || !std::isfinite(b.L))
    return set_err(c, UFC_ERR_ARG, "box side L must be finite and > 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(b.obs[a])) return set_err(c, UFC_ERR_ARG, "observer must be finite");
  if (b.shell_lo < 0 || b.shell_hi > nshell || b.shell_lo >= b.shell_hi)
    return set_err(c, UFC_ERR_ARG, "box shells [%d,%d) outside [0,%d)", b.shell_lo,
                   b.shell_hi, nshell);
  if (b.replicate < 0 || b.replicate > UFC_MAX_REPLICATE)
    return set_err(c, UFC_ERR_ARG, "replicate must be in [0,%d]", UFC_MAX_REPLICATE);
  g.shell_lo = b.shell_lo;
  g.shell_hi = b.shell_hi;
  g.R = b.replicate;
  const int n1 = 2 * b.replicate + 1;
  g.nimg = n1 * n1 * n1;
  float smax = 0.f;
  for (int a = 0; a < 3; ++a)
    for (int i = -b.replicate; i <= b.replicate; ++i) {
      double s = (double)i * b.L - b.obs[a];     // fl(fl(i L) - o)
      float hi = (float)s;
      float lo = (float)(s - (double)hi);
      g.sh64[a][i + b.replicate] = s;
      g.shf[a][i + b.replicate] = hi;
      g.shlo[a][i + b.replicate] = lo;
      smax = std::max(smax, std::fabs(hi));
    }
  g.smax = smax;
  return UFC_OK;
}

struct BinPlan {
  int mode;
  int shell0, shell1;            // shells any box of the call owns: [shell0, shell1)
  int nblk, nbuckets, ng, smem_hist;
};

// Particles per staged chunk of ufc_bin_host (402 MB); a multiple of 4, so
// that every chunk starts 16-byte aligned for the bulk copies.
constexpr int64_t kHostChunk = 1ll << 25;

// Workspace of one binning call of total_img particle images in
// fast_launches fast-stage launches.  Every warp of every launch (fast,
// refine, exact) may leave one partly filled queue chunk and one partly
// filled dense chunk behind.
struct BinSizes {
  int64_t cap1, cap2;   // queue slots
  int64_t dense_cap;    // dense key slots
  int64_t nb, ng;       // buckets and bucket groups of the dense path
};

static BinSizes bin_sizes(const ufc_ctx* c, int64_t fast_launches, int64_t total_img,
                          int nshell, int nside) {
  BinSizes z{};
  const int64_t fast_warps = (int64_t)std::max(2 * kFastThreads / 32, kWWarps) * c->num_sms;
  const int64_t late_warps = 2ll * 4 * c->num_sms * (256 / 32);
  const int64_t warps = fast_launches * fast_warps + late_warps + 64;
  z.cap1 = std::max<int64_t>(1 << 20, total_img / 16) + warps * kQChunk;
  z.cap2 = std::max<int64_t>(1 << 16, z.cap1 / 64) + warps * kQChunk;
  z.dense_cap = total_img + z.cap1 + warps * kChunk;
  const int64_t npix = 12ll * nside * nside;
  z.nb = nshell * (npix / kBlockPix);
  z.ng = (z.nb + (1 << kGroupBits) - 1) >> kGroupBits;
  return z;
}

// Grows the workspace for a binning call of total_img particle images at
// (nside, nshell) in fast_launches fast-stage launches (one per non-empty
// box for device input), so that the call itself allocates nothing.
ufc_status reserve_bin_workspace(ufc_ctx* c, int64_t fast_launches, int64_t total_img,
                                 int nshell, int nside) {
  const int64_t npix = 12ll * nside * nside;
  const BinSizes z = bin_sizes(c, fast_launches, total_img, nshell, nside);
  if (!ws_get(c, kSlotQueue1, z.cap1 * 8) || !ws_get(c, kSlotQueue2, z.cap2 * 8) ||
      !ws_get(c, kSlotOvf, (size_t)((total_img + 31) / 32) * 4))   // overflow bits (bound)
    return UFC_ERR_ALLOC;
  if (nside >= 64 && npix * nshell * 4 > (32ll << 20) && z.nb < (1ll << 17)) {
    if (!ws_get(c, kSlotDense, z.dense_cap * 4) || !ws_get(c, kSlotGrouped, (z.dense_cap + 4) * 4) ||
        !ws_get(c, kSlotBucket16, z.dense_cap * 2) || !ws_get(c, kSlotHist, z.nb * 4) ||
        !ws_get(c, kSlotOff, (z.nb + 1) * 8) || !ws_get(c, kSlotCursors, (z.nb + z.ng + 1) * 8) ||
        !ws_get(c, kSlotTiles, (size_t)(z.dense_cap / kScatTile + z.ng + 1) * sizeof(Tile)))
      return UFC_ERR_ALLOC;
  }
  return UFC_OK;
}

static cudaEvent_t copy_event(ufc_ctx* c, size_t i) {
  while (c->copy_events.size() <= i) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    c->copy_events.push_back(e);
  }
  return c->copy_events[i];
}

// Shell table and box geometry of a batched call's boxes (the persistent
// batch kernel of stats.cu keys particles with the same stages).
ufc_status batch_geometry(ufc_ctx* c, const double* chi, int nshell, const ufc_box* boxes,
                          int nbox, ShellTable& st, BoxGeom* bg) {
  ufc_status s = make_table(c, chi, nshell, st);
  if (s) return s;
  for (int k = 0; k < nbox; ++k) {
    s = make_box(c, boxes[k], nshell, bg[k]);
    if (s) return s;
  }
  return UFC_OK;
}
void batch_bands(int nside, float smax, Bands& bd) { make_bands(nside, smax, bd); }

// Runs the key pipeline for nbox boxes.  counts (DIRECT/DENSE) or keys (KEYS).
// xyz_host (non-NULL, ufc_bin_host): positions in host memory, copied into
// the staging slot chunk by chunk on the copy stream while the fast stage of
// the chunks already copied runs; xyz is then ignored.
ufc_status run_keys_pipeline(ufc_ctx* c, int mode_req, const float* const* xyz,
                             const int64_t* n, const ufc_box* boxes, int nbox,
                             const double* chi, int nshell, int nside, int flags,
                             int32_t* counts, int32_t* keys, const float* const* xyz_host) {
  if (nbox < 1 || nbox > kMaxBoxes)
    return set_err(c, UFC_ERR_ARG, "nbox must be in [1,%d]", kMaxBoxes);
  if (nshell < 1 || nshell > kMaxShells)
    return set_err(c, UFC_ERR_ARG, "nshell must be in [1,%d]", kMaxShells);
  if (nside < 1 || nside > UFC_MAX_NSIDE || (nside & (nside - 1)))
    return set_err(c, UFC_ERR_ARG, "nside must be a power of two in [1,%d]", UFC_MAX_NSIDE);
  const int64_t npix = 12ll * nside * nside;
  // keys shell * npix + pix are int32 (negative values mark outside/invalid)
  if ((int64_t)nshell * npix >= (1ll << 31))
    return set_err(c, UFC_ERR_ARG, "nshell * 12 nside^2 must be < 2^31");
  ShellTable st;
  ufc_status s = make_table(c, chi, nshell, st);
  if (s) return s;
  const float* staged[kMaxBoxes] = {};
  int64_t fast_launches = 0;
  if (xyz_host) {
    size_t total = 0;
    size_t offs[kMaxBoxes];
    for (int k = 0; k < nbox; ++k) {
      if (n[k] < 0) return set_err(c, UFC_ERR_ARG, "n[%d] < 0", k);
      if (n[k] > 0 && !xyz_host[k]) return set_err(c, UFC_ERR_ARG, "xyz_host[%d] is NULL", k);
      if (n[k] >= (1ll << 47)) return set_err(c, UFC_ERR_ARG, "n[%d] too large", k);
      offs[k] = total;
      total += ((size_t)n[k] * 12 + 255) & ~(size_t)255;
      fast_launches += (n[k] + kHostChunk - 1) / kHostChunk;
    }
    char* stage = (char*)ws_get(c, kSlotStage, total);
    if (!stage) return UFC_ERR_ALLOC;
    for (int k = 0; k < nbox; ++k) staged[k] = reinterpret_cast<const float*>(stage + offs[k]);
    xyz = staged;
  } else {
    for (int k = 0; k < nbox; ++k) fast_launches += n[k] > 0;
  }
  BoxesParam bp;
  std::memset(&bp, 0, sizeof bp);
  int64_t total_img = 0;
  float smax = 0.f;
  int maxR = 0;
  for (int k = 0; k < nbox; ++k) {
    if (n[k] < 0) return set_err(c, UFC_ERR_ARG, "n[%d] < 0", k);
    if (n[k] > 0 && !xyz[k]) return set_err(c, UFC_ERR_ARG, "xyz[%d] is NULL", k);
    if (n[k] >= (1ll << 47)) return set_err(c, UFC_ERR_ARG, "n[%d] too large", k);
    if (n[k] > 0 && (reinterpret_cast<uintptr_t>(xyz[k]) & 3))
      return set_err(c, UFC_ERR_ARG, "xyz[%d] is not 4-byte aligned", k);
    s = make_box(c, boxes[k], nshell, bp.box[k]);
    if (s) return s;
    bp.xyz[k] = xyz[k];
    bp.n[k] = n[k];
    total_img += n[k] * bp.box[k].nimg;
    smax = std::max(smax, bp.box[k].smax);
    maxR = std::max(maxR, (int)boxes[k].replicate);
  }
  Bands bd;
  make_bands(nside, smax, bd);

  BinPlan plan{};
  plan.mode = mode_req;
  plan.shell0 = nshell;
  plan.shell1 = 0;
  for (int k = 0; k < nbox; ++k) {
    plan.shell0 = std::min(plan.shell0, (int)boxes[k].shell_lo);
    plan.shell1 = std::max(plan.shell1, (int)boxes[k].shell_hi);
  }
  const int nwin = plan.shell1 - plan.shell0;   // the dense path covers these shells only
  if (mode_req != kModeKeys) {
    const int64_t map_bytes = (int64_t)nwin * npix * 4;
    const bool dense_ok = nside >= 64 && maxR == 0 &&
                          (int64_t)nwin * (npix / kBlockPix) < (1ll << 17);
    const bool aligned = (reinterpret_cast<uintptr_t>(counts) & 15) == 0;
    plan.mode = (dense_ok && aligned && map_bytes > (32ll << 20)) ? kModeDense : kModeDirect;
    if (flags & UFC_BIN_FORCE_DIRECT) plan.mode = kModeDirect;
    if (flags & UFC_BIN_FORCE_DENSE) {
      if (!(dense_ok && aligned))
        return set_err(c, UFC_ERR_UNSUPPORTED,
                       "the dense path needs nside >= 64, no replication, 16-byte aligned counts "
                       "and (shells of the boxes) * 12 nside^2 / 24576 < 2^17");
      plan.mode = kModeDense;
    }
  }
  if (plan.mode == kModeDense) {
    plan.nblk = (int)(npix / kBlockPix);
    plan.nbuckets = nwin * plan.nblk;
    plan.ng = (plan.nbuckets + (1 << kGroupBits) - 1) >> kGroupBits;
    // bucket counters in shared memory when both fast kernels still fit
    const size_t fixed = sizeof(FastShared) + 1024;
    plan.smem_hist = plan.nbuckets <= kSmemHistMax &&
                     kWSmemBase + ((plan.nbuckets + 1) / 2) * 4 + fixed <= (size_t)c->smem_optin &&
                     (size_t)plan.nbuckets * 4 + fixed <= (size_t)c->smem_optin;
  }

  // workspace
  const BinSizes z = bin_sizes(c, fast_launches, total_img, nshell, nside);
  Queues qs;
  qs.cap1 = z.cap1;
  qs.cap2 = z.cap2;
  qs.q1 = (uint64_t*)ws_get(c, kSlotQueue1, z.cap1 * 8);
  qs.q2 = (uint64_t*)ws_get(c, kSlotQueue2, z.cap2 * 8);
  if (!qs.q1 || !qs.q2) return UFC_ERR_ALLOC;
  qs.cnt = (BinCounters*)c->counters;
  UFC_CUDA(c, cudaMemsetAsync(qs.cnt, 0, offsetof(BinCounters, timeouts), c->stream));
  // overflow bits: one per particle of the boxes without periodic images
  int64_t nbits = 0;
  for (int k = 0; k < nbox; ++k) {
    bp.bit_base[k] = nbits;
    if (bp.box[k].nimg == 1) nbits += n[k];
  }
  const int64_t ovf_words = (nbits + 31) / 32;
  qs.ovf = (uint32_t*)ws_get(c, kSlotOvf, (size_t)ovf_words * 4);
  if (!qs.ovf) return UFC_ERR_ALLOC;
  qs.ovf_base = 0;
  if (ovf_words) UFC_CUDA(c, cudaMemsetAsync(qs.ovf, 0, (size_t)ovf_words * 4, c->stream));

  KeyOut o;
  std::memset(&o, 0, sizeof o);
  o.keys = keys;
  o.counts = counts;
  o.ncell = (int64_t)nshell * npix;
  o.dense_count = &qs.cnt->dense;
  int smem = 0;
  if (plan.mode == kModeDense) {
    o.dense_cap = z.dense_cap;
    o.dense = (uint32_t*)ws_get(c, kSlotDense, o.dense_cap * 4);
    o.hist = (uint32_t*)ws_get(c, kSlotHist, (size_t)plan.nbuckets * 4);
    if (!o.dense || !o.hist) return UFC_ERR_ALLOC;
    o.nblk = plan.nblk;
    o.nbuckets = plan.nbuckets;
    o.smem_hist = plan.smem_hist;
    o.shell0 = plan.shell0;
    UFC_CUDA(c, cudaMemsetAsync(o.hist, 0, (size_t)plan.nbuckets * 4, c->stream));
    if (!(flags & UFC_BIN_ACCUMULATE)) {   // shells outside the window hold no particle
      if (plan.shell0 > 0)
        UFC_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)plan.shell0 * npix * 4, c->stream));
      if (plan.shell1 < nshell)
        UFC_CUDA(c, cudaMemsetAsync(counts + (int64_t)plan.shell1 * npix, 0,
                                    (size_t)(nshell - plan.shell1) * npix * 4, c->stream));
    }
    smem = plan.smem_hist ? plan.nbuckets * 4 : 0;
  } else if (plan.mode == kModeDirect) {
    if (!(flags & UFC_BIN_ACCUMULATE))
      UFC_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)nshell * npix * 4, c->stream));
  }
  // shell lookup table over r^2: lut[i] = edges with lo2 <= i / scale
  LutParam lp;
  {
    // bins 0 .. kLut-2 cover [0, hi2[nshell]]
    const double top = std::max((double)st.hi2[nshell], 1e-30);
    lp.scale = (float)std::min((kLut - 2) / top, 1e30);
    const double sc = (double)lp.scale;
    int e0 = 0;
    for (int i = 0; i < kLut; ++i) {
      // r2 whose fminf(r2 * scale, kLut - 1) rounds to i has r2 * scale in
      // [i - 1/2, i + 1/2] up to the product's rounding (< 2^-11 here);
      // the range is widened by 2^-10
      const double rlo = ((double)i - 0.5 - 0x1p-10) / sc;
      const double rhi = (i == kLut - 1) ? INFINITY : ((double)i + 0.5 + 0x1p-10) / sc;
      while (e0 <= nshell && (double)st.hi2[e0] <= rlo) ++e0;
      const bool clean = e0 > nshell || (double)st.lo2[e0] > rhi;
      lp.v[i] = (uint16_t)(e0 | (clean ? 0 : kLutScan));
    }
  }
  // fast stage: one launch per box, or per staged chunk for host input
  const int tma_smem = kWSmemBase +
                       (plan.mode == kModeDense && plan.smem_hist ? ((plan.nbuckets + 1) / 2) * 4 : 0);
  if (xyz_host) {
    if (!c->copy_stream)
      UFC_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    // the copies overwrite the staging slot only after the work already on
    // the context stream (which may still read it) has finished
    cudaEvent_t e0 = copy_event(c, 0);
    if (!e0) return set_err(c, UFC_ERR_CUDA, "cudaEventCreate failed");
    UFC_CUDA(c, cudaEventRecord(e0, c->stream));
    UFC_CUDA(c, cudaStreamWaitEvent(c->copy_stream, e0, 0));
  }
  size_t nev = 1;
  for (int k = 0; k < nbox; ++k) {
    const int64_t step = xyz_host ? kHostChunk : std::max<int64_t>(n[k], 1);
    for (int64_t p0 = 0; p0 < n[k]; p0 += step) {
      const int64_t cnt = std::min(step, n[k] - p0);
      const float* src = xyz[k] + 3 * p0;
      if (xyz_host) {
        UFC_CUDA(c, cudaMemcpyAsync(const_cast<float*>(src), xyz_host[k] + 3 * p0,
                                    (size_t)cnt * 12, cudaMemcpyHostToDevice, c->copy_stream));
        cudaEvent_t e = copy_event(c, nev++);
        if (!e) return set_err(c, UFC_ERR_CUDA, "cudaEventCreate failed");
        UFC_CUDA(c, cudaEventRecord(e, c->copy_stream));
        UFC_CUDA(c, cudaStreamWaitEvent(c->stream, e, 0));
      }
      const bool tma = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
      ProfScope ps_(c, "k_fast");
      if (tma) {
        qs.ovf_base = bp.bit_base[k];
        const bool images = bp.box[k].nimg > 1;
#define UFC_LAUNCH_TMA(M, I)                                                                    \
  UFC_CUDA(c, cudaFuncSetAttribute(k_fast_tma<M, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   tma_smem));                                                   \
  k_fast_tma<M, I><<<c->num_sms, kWThreads, tma_smem, c->stream>>>(                              \
      src, cnt, p0, k, bp.box[k], st, lp, bd, nside, (int32_t)npix, o, qs)
        if (plan.mode == kModeDense) {
          if (images) { UFC_LAUNCH_TMA(kModeDense, true); } else { UFC_LAUNCH_TMA(kModeDense, false); }
        } else if (plan.mode == kModeDirect) {
          if (images) { UFC_LAUNCH_TMA(kModeDirect, true); } else { UFC_LAUNCH_TMA(kModeDirect, false); }
        } else {
          if (images) { UFC_LAUNCH_TMA(kModeKeys, true); } else { UFC_LAUNCH_TMA(kModeKeys, false); }
        }
#undef UFC_LAUNCH_TMA
      } else {
        const int ssm = plan.mode == kModeDense ? smem : 0;
#define UFC_LAUNCH_PLAIN(M)                                                                      \
  UFC_CUDA(c, cudaFuncSetAttribute(k_fast<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm)); \
  k_fast<M><<<(ssm > 0 ? 1 : 2) * c->num_sms, kFastThreads, ssm, c->stream>>>(                     \
      src, cnt, p0, k, bp.box[k], st, lp, bd, nside, (int32_t)npix, o, qs)
        if (plan.mode == kModeDense) { UFC_LAUNCH_PLAIN(kModeDense); }
        else if (plan.mode == kModeDirect) { UFC_LAUNCH_PLAIN(kModeDirect); }
        else { UFC_LAUNCH_PLAIN(kModeKeys); }
#undef UFC_LAUNCH_PLAIN
      }
      UFC_CUDA(c, cudaGetLastError());
    }
  }
  const int lgrid = 4 * c->num_sms;
  if (plan.mode == kModeDense) {
    {
      ProfScope ps_(c, "k_refine");
      k_refine<kModeDense><<<lgrid, 256, 0, c->stream>>>(bp, st, nside, (int32_t)npix, o, qs);
    }
    {
      ProfScope ps_(c, "k_exact");
      k_exact<kModeDense><<<lgrid, 256, 0, c->stream>>>(bp, st, nside, (int32_t)npix, o, qs);
    }
    if (ovf_words) {
      ProfScope ps_(c, "k_overflow");
      k_overflow<kModeDense><<<lgrid, 256, 0, c->stream>>>(bp, nbox, st, nside, (int32_t)npix, o, qs,
                                                      ovf_words);
    }
  } else if (plan.mode == kModeDirect) {
    {
      ProfScope ps_(c, "k_refine");
      k_refine<kModeDirect><<<lgrid, 256, 0, c->stream>>>(bp, st, nside, (int32_t)npix, o, qs);
    }
    {
      ProfScope ps_(c, "k_exact");
      k_exact<kModeDirect><<<lgrid, 256, 0, c->stream>>>(bp, st, nside, (int32_t)npix, o, qs);
    }
    if (ovf_words) {
      ProfScope ps_(c, "k_overflow");
      k_overflow<kModeDirect><<<lgrid, 256, 0, c->stream>>>(bp, nbox, st, nside, (int32_t)npix, o, qs,
                                                      ovf_words);
    }
  } else {
    {
      ProfScope ps_(c, "k_refine");
      k_refine<kModeKeys><<<lgrid, 256, 0, c->stream>>>(bp, st, nside, (int32_t)npix, o, qs);
    }
    {
      ProfScope ps_(c, "k_exact");
      k_exact<kModeKeys><<<lgrid, 256, 0, c->stream>>>(bp, st, nside, (int32_t)npix, o, qs);
    }
    if (ovf_words) {
      ProfScope ps_(c, "k_overflow");
      k_overflow<kModeKeys><<<lgrid, 256, 0, c->stream>>>(bp, nbox, st, nside, (int32_t)npix, o, qs,
                                                      ovf_words);
    }
  }
  UFC_CUDA(c, cudaGetLastError());
  if (plan.mode != kModeDense) return UFC_OK;

  // ---- dense pipeline: scan, two scatter passes, per-bucket histograms ----
  const int nb = plan.nbuckets, ng = plan.ng;
  int64_t* off = (int64_t*)ws_get(c, kSlotOff, (size_t)(nb + 1) * 8);
  unsigned long long* cur = (unsigned long long*)ws_get(c, kSlotCursors, (size_t)(nb + ng + 1) * 8);
  // 4 keys of slack: a tile's bulk copy ends at the 16-byte unit holding its last key
  uint32_t* grouped = (uint32_t*)ws_get(c, kSlotGrouped, (size_t)(o.dense_cap + 4) * 4);
  uint16_t* b16 = (uint16_t*)ws_get(c, kSlotBucket16, (size_t)o.dense_cap * 2);
  const int64_t max_tiles = o.dense_cap / kScatTile + ng + 1;
  Tile* tiles = (Tile*)ws_get(c, kSlotTiles, (size_t)max_tiles * sizeof(Tile));
  if (!off || !cur || !grouped || !b16 || !tiles) return UFC_ERR_ALLOC;
  unsigned long long* gcur = cur;
  unsigned long long* bcur = cur + ng;
  unsigned long long* ntiles = &qs.cnt->ntiles;
  {
    ProfScope ps_(c, "k_scan");
    k_scan<<<1, 1024, 0, c->stream>>>(o.hist, nb, off);
  }
  {
    ProfScope ps_(c, "k_cursors");
    k_cursors<<<(std::max(nb, ng) + 255) / 256, 256, 0, c->stream>>>(off, nb, ng, gcur, bcur);
  }
  const int smemA = 2 * (kScatTile + 4) * 4 + kScatTile * 4 + ng * 16;
  UFC_CUDA(c, cudaFuncSetAttribute(k_scatter_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smemA));
  {
    ProfScope ps_(c, "k_scatter_group");
    k_scatter_group<<<2 * c->num_sms, kScatThreads, smemA, c->stream>>>(
        o.dense, o.dense_count, o.dense_cap, ng, gcur, grouped, &qs.cnt->timeouts);
  }
  {
    ProfScope ps_(c, "k_tiles");
    k_tiles<<<c->num_sms, kTilesThreads, (size_t)(2 * ng + 2) * 8, c->stream>>>(off, nb, ng, tiles,
                                                                              ntiles);
  }
  const int smemB = 2 * (kScatTile + 4) * 4 + (1 << kGroupBits) * 16 + kScatTile * 4;
  UFC_CUDA(c, cudaFuncSetAttribute(k_scatter_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smemB));
  {
    ProfScope ps_(c, "k_scatter_bucket");
    k_scatter_bucket<<<2 * c->num_sms, kScatThreads, smemB, c->stream>>>(
        grouped, tiles, ntiles, bcur, b16, o.dense_cap, &qs.cnt->timeouts);
  }
  const int smemH = kBlockPix * 4;
  UFC_CUDA(c, cudaFuncSetAttribute(k_hist_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smemH));
  {
    ProfScope ps_(c, "k_hist_block");
    k_hist_block<<<2 * c->num_sms, kHistThreads, smemH, c->stream>>>(
        b16, off, nb, counts + (int64_t)plan.shell0 * npix, (flags & UFC_BIN_ACCUMULATE) ? 1 : 0,
        o.dense_cap);
  }
  UFC_CUDA(c, cudaGetLastError());
  return UFC_OK;
}

}  // namespace ufc

namespace ufc {

// Binning from host memory through a bounded device buffer: the boxes'
// particles are cut into chunks of at most `chunk` particles; chunk i+1 is
// copied into one of two device buffers on the copy stream while chunk i is
// binned from the other on the context stream.  Every chunk is a complete
// binning call into counts (accumulating after the first), so the device
// memory held is two chunks plus one chunk's workspace whatever the
// particle count.
ufc_status run_bin_stream(ufc_ctx* c, const float* const* xyz_host, const int64_t* n,
                          const ufc_box* boxes, int nbox, const double* chi, int nshell,
                          int nside, int flags, int64_t chunk, int32_t* counts) {
  if (nbox < 1 || nbox > kMaxBoxes) return set_err(c, UFC_ERR_ARG, "nbox must be in [1,%d]", kMaxBoxes);
  if (chunk < 1) return set_err(c, UFC_ERR_ARG, "chunk must be >= 1");
  int64_t largest = 0;
  for (int k = 0; k < nbox; ++k) {
    if (n[k] < 0) return set_err(c, UFC_ERR_ARG, "n[%d] < 0", k);
    if (n[k] > 0 && !xyz_host[k]) return set_err(c, UFC_ERR_ARG, "xyz_host[%d] is NULL", k);
    largest = std::max(largest, std::min(n[k], chunk));
  }
  const size_t bufb = ((size_t)largest * 12 + 255) & ~(size_t)255;
  char* stage = (char*)ws_get(c, kSlotStage, 2 * std::max<size_t>(bufb, 256));
  if (!stage) return UFC_ERR_ALLOC;
  float* buf[2] = {reinterpret_cast<float*>(stage), reinterpret_cast<float*>(stage + bufb)};
  if (!c->copy_stream)
    UFC_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  // events: 0, 1 = buffer free; 2, 3 = buffer filled
  for (int i = 0; i < 4; ++i)
    if (!copy_event(c, i)) return set_err(c, UFC_ERR_CUDA, "cudaEventCreate failed");
  for (int b = 0; b < 2; ++b) UFC_CUDA(c, cudaEventRecord(c->copy_events[b], c->stream));
  bool first = !(flags & UFC_BIN_ACCUMULATE);
  int it = 0;
  for (int k = 0; k < nbox; ++k) {
    for (int64_t p0 = 0; p0 < n[k]; p0 += chunk, ++it) {
      const int64_t cnt = std::min(chunk, n[k] - p0);
      const int b = it & 1;
      UFC_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->copy_events[b], 0));
      UFC_CUDA(c, cudaMemcpyAsync(buf[b], xyz_host[k] + 3 * p0, (size_t)cnt * 12,
                                  cudaMemcpyHostToDevice, c->copy_stream));
      UFC_CUDA(c, cudaEventRecord(c->copy_events[2 + b], c->copy_stream));
      UFC_CUDA(c, cudaStreamWaitEvent(c->stream, c->copy_events[2 + b], 0));
      const float* xs[1] = {buf[b]};
      const int fl = (flags & (UFC_BIN_FORCE_DIRECT | UFC_BIN_FORCE_DENSE)) |
                     (first ? 0 : UFC_BIN_ACCUMULATE);
      ufc_status s = run_keys_pipeline(c, 1, xs, &cnt, &boxes[k], 1, chi, nshell, nside, fl,
                                       counts, nullptr, nullptr);
      if (s) return s;
      UFC_CUDA(c, cudaEventRecord(c->copy_events[b], c->stream));
      first = false;
    }
  }
  if (first && !(flags & UFC_BIN_ACCUMULATE)) {      // no particles at all: zero counts
    UFC_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)nshell * 12 * nside * nside * 4, c->stream));
  }
  return UFC_OK;
}

}  // namespace ufc
