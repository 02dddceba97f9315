// Library context and device workspace (internal).
#pragma once
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/ufalcon.h"

struct ufc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int num_sms = 0;
  int smem_optin = 0;            // shared memory per block with opt-in (bytes)
  // grow-only device buffers, one per slot
  static constexpr int kSlots = 18;
  void* buf[kSlots] = {};
  size_t cap[kSlots] = {};
  void* counters = nullptr;      // ufc::BinCounters of the last binning call
  // kernel timing: events bracketing each launch while enabled
  bool prof = false;
  struct ProfRec { const char* name; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_pool_used = 0;
  // binning from host memory: a copy stream and one event per staged chunk
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> copy_events;
  // graph capture when the caller's stream is the legacy default stream:
  // captured on aux_stream, forked and joined by aux_ev
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
  // executable graph of the last ufc_batched_stats call with UFC_BATCH_GRAPH
  // and that call's host arguments, byte for byte; dropped whenever a
  // workspace buffer it refers to is reallocated
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  // ufc_batched_stats on small maps: extra contexts ("lanes") with their
  // own workspace, counters and stream, each binning a share of the
  // realisations concurrently; a lane's owner drops its graph whenever the
  // lane's workspace is reallocated
  static constexpr int kMaxLanes = 8;
  ufc_ctx* lanes[kMaxLanes] = {};
  cudaStream_t lane_stream[kMaxLanes] = {};
  cudaEvent_t lane_ev[kMaxLanes + 1] = {};
  ufc_ctx* owner = nullptr;
  // tuning (ufc_set_tuning) and the prepared launch of the persistent
  // batch kernel (descriptors uploaded, launch arguments kept here)
  int32_t batch_chunk = 0, batch_blocks_per_sm = 0;
  std::vector<unsigned char> batch_launch;
};

namespace ufc {

enum Slot {
  kSlotQueue1 = 0,
  kSlotQueue2,
  kSlotDense,
  kSlotGrouped,
  kSlotBucket16,
  kSlotHist,
  kSlotOff,
  kSlotCursors,
  kSlotTiles,
  kSlotPartials,
  kSlotCoeffs,
  kSlotMisc,
  kSlotStage,      // device copy of host particle positions (ufc_bin_host)
  kSlotSht,        // ring transforms, Legendre seeds, partial a_lm (ufc_map2alm)
  kSlotOvf,        // one bit per particle image: left undecided when queue 1 was full
  kSlotLaneMap,    // a lane's count map and kappa map (ufc_batched_stats)
  kSlotBatchMaps,  // persistent batch kernel: per-realisation maps and partial sums
  kSlotBatchDesc,  // persistent batch kernel: task descriptors and queue counters
};

inline ufc_status set_err(ufc_ctx* c, ufc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define UFC_CUDA(c, call)                                                       \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return ::ufc::set_err((c), UFC_ERR_CUDA, "%s: %s (%s:%d)", #call,         \
                            cudaGetErrorString(e_), __FILE__, __LINE__);        \
  } while (0)

// Kernel timing and tracing.  prof_begin/prof_end bracket one launch on the
// context's stream with CUDA events when timing is enabled
// (ufc_profile_enable).  Every launch is also an NVTX range named after its
// kernel (header-only NVTX 3: a no-op unless a tool such as Nsight Systems
// is attached), so a timeline shows the library's steps.
void prof_begin(ufc_ctx* c, const char* name);
void prof_end(ufc_ctx* c);

struct ProfScope {
  ufc_ctx* c;
  ProfScope(ufc_ctx* c_, const char* name) : c(c_) {
    nvtxRangePushA(name);
    prof_begin(c, name);
  }
  ~ProfScope() {
    prof_end(c);
    nvtxRangePop();
  }
};

// Ensures slot `s` holds at least `bytes`; returns nullptr (and sets the
// error) when the allocation fails.  Growing frees the old buffer, which
// waits for the device.
void* ws_get(ufc_ctx* c, int s, size_t bytes);

}  // namespace ufc
