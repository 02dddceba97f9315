// C ABI of libufalcon_gb300.so: argument checks, context, workspace, and the
// calls into the binning, statistics and cosmology code.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace ufc {
ufc_status run_keys_pipeline(ufc_ctx* c, int mode_req, const float* const* xyz,
                             const int64_t* n, const ufc_box* boxes, int nbox,
                             const double* chi, int nshell, int nside, int flags,
                             int32_t* counts, int32_t* keys, const float* const* xyz_host);
ufc_status run_kappa_stats(ufc_ctx* c, const int32_t* counts, int S, int nside,
                           const double* A, double C, double lo, double hi, int nbins,
                           float* kappa, double* moments, int64_t* pdf);
ufc_status run_kappa_backward(ufc_ctx* c, const int32_t* counts, int S, int nside,
                              const double* A, double C, double w_var, double w_skew,
                              const float* g, const double* dA, const double* dC,
                              double* grad, double* G, double* H);
ufc_status run_kappa_backward_ex(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                 const double* A, double C, double w_var, double w_skew,
                                 const float* g, const double* dA, const double* dC,
                                 double* grad, double* G, double* H, float* kappa, double lo,
                                 double hi, int nbins, double* moments, int64_t* pdf);
ufc_status run_kappa_partial(ufc_ctx* c, const int32_t* counts, int S, int nside,
                             const double* A, double* partial);
ufc_status run_kappa_stats_partial(ufc_ctx* c, const double* partial, int nside, double C,
                                   double lo, double hi, int nbins, float* kappa,
                                   double* moments, int64_t* pdf);
ufc_status run_kappa_adjoint_sums(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                  const double* partial, double C, const float* g, float* kappa,
                                  double lo, double hi, int nbins, double* moments, int64_t* pdf,
                                  double* sums);
void grad_from_sums(const double* sm, int S, int npix, double w_var, double w_skew,
                    const double* dA, const double* dC, double* grad, double* G, double* H);
cudaError_t take_checks_bin(CheckRec* out, cudaStream_t s);
cudaError_t take_checks_stats(CheckRec* out, cudaStream_t s);
ufc_status run_check_selftest(ufc_ctx* c, int64_t index, int64_t bound);
ufc_status run_welford_update(ufc_ctx* c, const double* v, int nvec, int d, double* st);
ufc_status run_stats_vector(ufc_ctx* c, const double* m, const int64_t* pdf, int nbins, double* v);
ufc_status run_kappa_stats_noalloc(ufc_ctx* c, const int32_t* counts, int S, int nside,
                                   const double* A, double C, double lo, double hi, int nbins,
                                   float* kappa, double* moments, int64_t* pdf);
ufc_status run_welford_merge(ufc_ctx* c, double* a, const double* b, int d);
void batch_persistent_bytes(const ufc_ctx* c, int nreal, int nbox, int S, int nside,
                            size_t* maps, size_t* desc);
ufc_status batch_persistent_prepare(ufc_ctx* c, int nreal, int nbox, const float* const* xyz,
                                    const int64_t* n, const ufc_box* boxes, const double* chi,
                                    int S, int nside, const double* A, const double* C, double lo,
                                    double hi, int nbins, double* moments, int64_t* pdf,
                                    double* stats, double* state, char* maps, char* desc);
ufc_status batch_persistent_enqueue(ufc_ctx* c, char* maps, char* desc);
ufc_status run_welford_finalize(ufc_ctx* c, const double* st, int d, int ddof, double* mean,
                                double* cov, double* corr);
ufc_status reserve_bin_workspace(ufc_ctx* c, int64_t fast_launches, int64_t total_img,
                                 int nshell, int nside);
ufc_status run_map2alm(ufc_ctx* c, const float* map, int nside, int lmax, double* alm_out);
ufc_status run_alm2cl(ufc_ctx* c, const double* alm, int lmax, double* cl);
ufc_status run_cl_bin(ufc_ctx* c, const double* cl, int lmax, int lmin, int dl, int nbins,
                      double* out);
ufc_status run_alm2map(ufc_ctx* c, const double* alm, int nside, int lmax, float* map);
ufc_status run_wait_selftest(ufc_ctx* c, int64_t limit);
ufc_status run_bin_stream(ufc_ctx* c, const float* const* xyz_host, const int64_t* n,
                          const ufc_box* boxes, int nbox, const double* chi, int nshell,
                          int nside, int flags, int64_t chunk, int32_t* counts);
ufc_status run_alm_beam(ufc_ctx* c, const double* in, int lmax, double sigma, double* out);
ufc_status run_map_stats(ufc_ctx* c, const float* map, int nside, double lo, double hi,
                         int nbins, double* moments, int64_t* pdf);
ufc_status cosmo_chi_edges(const ufc_cosmo& c, const double* z, int n, double* chi);
ufc_status cosmo_z_of_chi(const ufc_cosmo& c, const double* chi, int n, double* zout);
ufc_status cosmo_kappa_coeffs(const ufc_cosmo& c, const ufc_box* boxes, int nbox,
                              const double* z, int S, int nside, const ufc_source& src,
                              double* A, double* B, double* C, double* dA, double* dC);
ufc_status cosmo_delta_coeffs(const ufc_cosmo& c, const ufc_box* boxes, int nbox,
                              const double* z, int S, int nside, double* A, double* C,
                              double* dA, double* dC);

void* ws_get(ufc_ctx* c, int s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (c->cap[s] >= bytes) return c->buf[s];
  if (c->buf[s]) {
    cudaStreamSynchronize(c->stream);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    if (c->aux_stream) cudaStreamSynchronize(c->aux_stream);
    ufc_ctx* gc = c->owner ? c->owner : c;   // the context whose graph may use this buffer
    if (gc->graph_exec) {                 // the cached graph refers to this buffer
      cudaStreamSynchronize(gc->stream);
      if (gc->aux_stream) cudaStreamSynchronize(gc->aux_stream);
      cudaGraphExecDestroy(gc->graph_exec);
      gc->graph_exec = nullptr;
      gc->graph_key.clear();
    }
    cudaFree(c->buf[s]);
    c->buf[s] = nullptr;
    c->cap[s] = 0;
  }
  size_t want = bytes + bytes / 8;   // some headroom against repeated growth
  if (cudaMalloc(&c->buf[s], want) != cudaSuccess) {
    cudaGetLastError();
    c->buf[s] = nullptr;
    set_err(c, UFC_ERR_ALLOC, "cudaMalloc of %zu bytes for workspace slot %d failed", want, s);
    return nullptr;
  }
  c->cap[s] = want;
  return c->buf[s];
}

static cudaEvent_t prof_event(ufc_ctx* c) {
  if (c->prof_pool_used == c->prof_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->prof_pool.push_back(e);
  }
  return c->prof_pool[c->prof_pool_used++];
}

void prof_begin(ufc_ctx* c, const char* name) {
  if (!c || !c->prof) return;
  cudaEvent_t a = prof_event(c), b = prof_event(c);
  if (!a || !b) return;
  cudaEventRecord(a, c->stream);
  c->prof_recs.push_back({name, a, b});
}

void prof_end(ufc_ctx* c) {
  if (!c || !c->prof || c->prof_recs.empty()) return;
  cudaEventRecord(c->prof_recs.back().b, c->stream);
}

static ufc_status check_cosmo(ufc_ctx* c, const ufc_cosmo* cs) {
  if (!cs) return set_err(c, UFC_ERR_ARG, "cosmo is NULL");
  if (!(cs->omega_m >= 0.0 && cs->omega_m <= 1.0))
    return set_err(c, UFC_ERR_ARG, "omega_m must be in [0,1]");
  if (!(cs->h > 0.0) || !std::isfinite(cs->h)) return set_err(c, UFC_ERR_ARG, "h must be > 0");
  if (cs->units_mpc_over_h != 0 && cs->units_mpc_over_h != 1)
    return set_err(c, UFC_ERR_ARG, "units_mpc_over_h must be 0 or 1");
  if (cs->density_volume != 0 && cs->density_volume != 1)
    return set_err(c, UFC_ERR_ARG, "density_volume must be 0 or 1");
  return UFC_OK;
}

static ufc_status check_z(ufc_ctx* c, const double* z, int n) {
  if (!z) return set_err(c, UFC_ERR_ARG, "z_edges is NULL");
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(z[i]) || z[i] < 0.0 || z[i] > 20.0)
      return set_err(c, UFC_ERR_ARG, "z_edges[%d] = %g outside [0,20]", i, z[i]);
    if (i && !(z[i] > z[i - 1])) return set_err(c, UFC_ERR_ARG, "z_edges must increase");
  }
  return UFC_OK;
}

}  // namespace ufc

using namespace ufc;

extern "C" {

ufc_status ufc_create(ufc_ctx** out, int32_t device) {
  if (!out) return UFC_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return UFC_ERR_CUDA;
  }
  ufc_ctx* c = new (std::nothrow) ufc_ctx();
  if (!c) return UFC_ERR_ALLOC;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete c; return UFC_ERR_CUDA; }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (cudaMalloc(&c->counters, sizeof(BinCounters)) != cudaSuccess) { delete c; return UFC_ERR_ALLOC; }
  cudaMemset(c->counters, 0, sizeof(BinCounters));
  *out = c;
  return UFC_OK;
}

ufc_status ufc_destroy(ufc_ctx* c) {
  if (!c) return UFC_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (int s = 0; s < ufc_ctx::kSlots; ++s)
    if (c->buf[s]) cudaFree(c->buf[s]);
  if (c->counters) cudaFree(c->counters);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (cudaEvent_t e : c->copy_events) cudaEventDestroy(e);
  if (c->aux_stream) {
    cudaStreamSynchronize(c->aux_stream);
    cudaStreamDestroy(c->aux_stream);
  }
  for (cudaEvent_t e : c->aux_ev)
    if (e) cudaEventDestroy(e);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  for (int k = 0; k < ufc_ctx::kMaxLanes; ++k) {
    if (c->lane_stream[k]) cudaStreamSynchronize(c->lane_stream[k]);
    if (c->lanes[k]) { c->lanes[k]->stream = c->lane_stream[k]; ufc_destroy(c->lanes[k]); }
    if (c->lane_stream[k]) cudaStreamDestroy(c->lane_stream[k]);
  }
  for (cudaEvent_t e : c->lane_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return UFC_OK;
}

ufc_status ufc_set_stream(ufc_ctx* c, void* stream) {
  if (!c) return UFC_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return UFC_OK;
}

ufc_status ufc_synchronize(ufc_ctx* c) {
  if (!c) return UFC_ERR_ARG;
  cudaSetDevice(c->device);
  // the timeouts of this context and of its batched lanes; each counter is
  // read and cleared on its own stream, after the work enqueued there
  unsigned long long t[ufc_ctx::kMaxLanes + 1] = {};
  ufc_ctx* owners[ufc_ctx::kMaxLanes + 1] = {c};
  int n = 1;
  for (int k = 0; k < ufc_ctx::kMaxLanes; ++k)
    if (c->lanes[k]) owners[n++] = c->lanes[k];
  for (int k = 0; k < n; ++k) {
    BinCounters* bc = reinterpret_cast<BinCounters*>(owners[k]->counters);
    UFC_CUDA(c, cudaMemcpyAsync(&t[k], &bc->timeouts, sizeof t[k], cudaMemcpyDeviceToHost,
                                owners[k]->stream));
    UFC_CUDA(c, cudaMemsetAsync(&bc->timeouts, 0, sizeof t[k], owners[k]->stream));
  }
  unsigned long long total = 0;
  for (int k = 0; k < n; ++k) {
    UFC_CUDA(c, cudaStreamSynchronize(owners[k]->stream));
    total += t[k];
  }
  // index-test records (per device and translation unit), after all the work
  CheckRec rec[2] = {};
  UFC_CUDA(c, take_checks_bin(&rec[0], c->stream));
  UFC_CUDA(c, take_checks_stats(&rec[1], c->stream));
  UFC_CUDA(c, cudaStreamSynchronize(c->stream));
  if (total)
    return set_err(c, UFC_ERR_TIMEOUT,
                   "%llu device-side bounded wait(s) ran out since the last report; the "
                   "binning calls that met them have incomplete counts", total);
  for (const CheckRec& r : rec)
    if (r.count)
      return set_err(c, UFC_ERR_INTERNAL,
                     "%llu index test(s) failed since the last report; first at site %lld: "
                     "index %lld, bound %lld (the accesses were skipped)",
                     r.count, r.site, r.index, r.bound);
  return UFC_OK;
}

ufc_status ufc_check_selftest(ufc_ctx* c, int64_t index, int64_t bound) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_check_selftest(c, index, bound);
}

ufc_status ufc_wait_selftest(ufc_ctx* c, int64_t limit) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_wait_selftest(c, limit);
}

const char* ufc_last_error(const ufc_ctx* c) { return c ? c->err.c_str() : "no context"; }

static int64_t held_bytes(const ufc_ctx* c) {
  int64_t t = c->counters ? (int64_t)sizeof(BinCounters) : 0;
  for (int s = 0; s < ufc_ctx::kSlots; ++s) t += (int64_t)c->cap[s];
  for (int k = 0; k < ufc_ctx::kMaxLanes; ++k)
    if (c->lanes[k]) t += held_bytes(c->lanes[k]);
  return t;
}

ufc_status ufc_workspace_bytes(const ufc_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return UFC_ERR_ARG;
  *bytes = held_bytes(c);
  return UFC_OK;
}

ufc_status ufc_set_tuning(ufc_ctx* c, const ufc_tuning* t) {
  if (!c || !t) return UFC_ERR_ARG;
  if (t->batch_chunk < 0 || t->batch_chunk > (1 << 24) || t->batch_blocks_per_sm < 0 ||
      t->batch_blocks_per_sm > 2)
    return set_err(c, UFC_ERR_ARG, "tuning out of range (chunk <= 2^24, blocks per SM <= 2)");
  c->batch_chunk = t->batch_chunk;
  c->batch_blocks_per_sm = t->batch_blocks_per_sm;
  return UFC_OK;
}

ufc_status ufc_get_tuning(const ufc_ctx* c, ufc_tuning* t) {
  if (!c || !t) return UFC_ERR_ARG;
  t->batch_chunk = c->batch_chunk;
  t->batch_blocks_per_sm = c->batch_blocks_per_sm;
  return UFC_OK;
}

ufc_status ufc_reserve(ufc_ctx* c, int32_t nside, int32_t nshell, int64_t n_max) {
  if (!c || nside < 1 || nshell < 1 || n_max < 0) return UFC_ERR_ARG;
  cudaSetDevice(c->device);
  return reserve_bin_workspace(c, 2, n_max, nshell, nside);
}

ufc_status ufc_profile_enable(ufc_ctx* c, int32_t on) {
  if (!c) return UFC_ERR_ARG;
  c->prof = on != 0;
  return UFC_OK;
}

ufc_status ufc_profile_read(ufc_ctx* c, int32_t max, char* names, double* ms,
                            int64_t* launches, int32_t* n_out) {
  if (!c || max < 0 || !n_out || (max > 0 && (!names || !ms || !launches))) return UFC_ERR_ARG;
  cudaSetDevice(c->device);
  UFC_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<std::string> keys;
  std::vector<double> tot;
  std::vector<int64_t> cnt;
  for (const auto& r : c->prof_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { cudaGetLastError(); continue; }
    size_t i = 0;
    while (i < keys.size() && keys[i] != r.name) ++i;
    if (i == keys.size()) { keys.push_back(r.name); tot.push_back(0.0); cnt.push_back(0); }
    tot[i] += t;
    cnt[i] += 1;
  }
  const int n = (int)keys.size();
  for (int i = 0; i < n && i < max; ++i) {
    std::memset(names + 32 * i, 0, 32);
    std::strncpy(names + 32 * i, keys[i].c_str(), 31);
    ms[i] = tot[i];
    launches[i] = cnt[i];
  }
  *n_out = n;
  c->prof_recs.clear();
  c->prof_pool_used = 0;
  return UFC_OK;
}

ufc_status ufc_chi_edges(const ufc_cosmo* cosmo, const double* z_edges, int32_t nshell,
                         double* chi_out) {
  ufc_status s = check_cosmo(nullptr, cosmo);
  if (s) return s;
  if (nshell < 1 || !chi_out) return UFC_ERR_ARG;
  s = check_z(nullptr, z_edges, nshell + 1);
  if (s) return s;
  return cosmo_chi_edges(*cosmo, z_edges, nshell + 1, chi_out);
}

ufc_status ufc_z_of_chi(const ufc_cosmo* cosmo, const double* chi, int32_t n, double* z_out) {
  ufc_status s = check_cosmo(nullptr, cosmo);
  if (s) return s;
  if (n < 0 || (n && (!chi || !z_out))) return UFC_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(chi[i]) || chi[i] < 0.0) return UFC_ERR_ARG;
  return cosmo_z_of_chi(*cosmo, chi, n, z_out);
}

// Arguments shared by the kappa and delta coefficient calls.
static ufc_status check_map_geometry(const ufc_cosmo* cosmo, const ufc_box* boxes, int32_t nbox,
                                     const double* z_edges, int32_t nshell, int32_t nside) {
  ufc_status s = check_cosmo(nullptr, cosmo);
  if (s) return s;
  if (!boxes || nbox < 1 || nshell < 1 || nshell > UFC_MAX_SHELLS) return UFC_ERR_ARG;
  if (nside < 1 || nside > UFC_MAX_NSIDE || (nside & (nside - 1))) return UFC_ERR_ARG;
  s = check_z(nullptr, z_edges, nshell + 1);
  if (s) return s;
  if (!(z_edges[0] > 0.0)) return UFC_ERR_ARG;   // Eq. 6 and 7 divide by chi(z_0)^2
  for (int b = 0; b < nshell; ++b) {
    int owners = 0;
    for (int k = 0; k < nbox; ++k)
      owners += (b >= boxes[k].shell_lo && b < boxes[k].shell_hi);
    if (owners != 1) return UFC_ERR_ARG;
  }
  for (int k = 0; k < nbox; ++k)
    if (!(boxes[k].L > 0.0) || boxes[k].n_total < 1) return UFC_ERR_ARG;
  return UFC_OK;
}

ufc_status ufc_delta_coeffs(const ufc_cosmo* cosmo, const ufc_box* boxes, int32_t nbox,
                            const double* z_edges, int32_t nshell, int32_t nside, double* A,
                            double* C, double* dA, double* dC) {
  ufc_status s = check_map_geometry(cosmo, boxes, nbox, z_edges, nshell, nside);
  if (s) return s;
  if (!A || !C) return UFC_ERR_ARG;
  return cosmo_delta_coeffs(*cosmo, boxes, nbox, z_edges, nshell, nside, A, C, dA, dC);
}

ufc_status ufc_kappa_coeffs(const ufc_cosmo* cosmo, const ufc_box* boxes, int32_t nbox,
                            const double* z_edges, int32_t nshell, int32_t nside,
                            const ufc_source* src, double* A, double* B, double* C,
                            double* dA, double* dC) {
  ufc_status s = check_map_geometry(cosmo, boxes, nbox, z_edges, nshell, nside);
  if (s) return s;
  if (!src || !A || !C) return UFC_ERR_ARG;
  if (src->kind == 0) {
    if (!(src->z_s > 0.0) || src->z_s > 20.0) return UFC_ERR_ARG;
  } else if (src->kind == 1) {
    if (!(src->z_max > 0.0) || src->z_max > 20.0 || !(src->z0 > 0.0) || !(src->beta > 0.0) ||
        !(src->alpha > -1.0))
      return UFC_ERR_ARG;
  } else {
    return UFC_ERR_ARG;
  }
  return cosmo_kappa_coeffs(*cosmo, boxes, nbox, z_edges, nshell, nside, *src, A, B, C, dA, dC);
}

ufc_status ufc_keys(ufc_ctx* c, const float* xyz_dev, int64_t n, const ufc_box* box,
                    const double* chi_edges, int32_t nshell, int32_t nside,
                    int32_t* keys_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!box || !chi_edges) return set_err(c, UFC_ERR_ARG, "box and chi_edges are required");
  if (n > 0 && !keys_dev) return set_err(c, UFC_ERR_ARG, "keys_dev is NULL");
  if (box->replicate != 0) return set_err(c, UFC_ERR_ARG, "ufc_keys needs replicate = 0");
  cudaSetDevice(c->device);
  return run_keys_pipeline(c, 0, &xyz_dev, &n, box, 1, chi_edges, nshell, nside, 0, nullptr,
                           keys_dev, nullptr);
}

ufc_status ufc_bin(ufc_ctx* c, const float* const* xyz_dev, const int64_t* n,
                   const ufc_box* boxes, int32_t nbox, const double* chi_edges,
                   int32_t nshell, int32_t nside, int32_t flags, int32_t* counts_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!xyz_dev || !n || !boxes || !chi_edges || !counts_dev)
    return set_err(c, UFC_ERR_ARG, "NULL argument to ufc_bin");
  if (flags & ~(UFC_BIN_ACCUMULATE | UFC_BIN_FORCE_DIRECT | UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "unknown flags");
  if ((flags & UFC_BIN_FORCE_DIRECT) && (flags & UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "FORCE_DIRECT and FORCE_DENSE exclude each other");
  if (reinterpret_cast<uintptr_t>(counts_dev) & 3)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 4-byte aligned");
  cudaSetDevice(c->device);
  return run_keys_pipeline(c, 1, xyz_dev, n, boxes, nbox, chi_edges, nshell, nside, flags,
                           counts_dev, nullptr, nullptr);
}

ufc_status ufc_bin_host(ufc_ctx* c, const float* const* xyz_host, const int64_t* n,
                        const ufc_box* boxes, int32_t nbox, const double* chi_edges,
                        int32_t nshell, int32_t nside, int32_t flags, int32_t* counts_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!xyz_host || !n || !boxes || !chi_edges || !counts_dev)
    return set_err(c, UFC_ERR_ARG, "NULL argument to ufc_bin_host");
  if (flags & ~(UFC_BIN_ACCUMULATE | UFC_BIN_FORCE_DIRECT | UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "unknown flags");
  if ((flags & UFC_BIN_FORCE_DIRECT) && (flags & UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "FORCE_DIRECT and FORCE_DENSE exclude each other");
  if (reinterpret_cast<uintptr_t>(counts_dev) & 3)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 4-byte aligned");
  cudaSetDevice(c->device);
  cudaStreamCaptureStatus cs;
  UFC_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return set_err(c, UFC_ERR_UNSUPPORTED, "ufc_bin_host cannot be captured into a graph");
  return run_keys_pipeline(c, 1, nullptr, n, boxes, nbox, chi_edges, nshell, nside, flags,
                           counts_dev, nullptr, xyz_host);
}

ufc_status ufc_map2alm(ufc_ctx* c, const float* map_dev, int32_t nside, int32_t lmax,
                       double* alm_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_map2alm(c, map_dev, nside, lmax, alm_dev);
}

ufc_status ufc_alm2cl(ufc_ctx* c, const double* alm_dev, int32_t lmax, double* cl_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_alm2cl(c, alm_dev, lmax, cl_dev);
}

ufc_status ufc_cl_bin(ufc_ctx* c, const double* cl_dev, int32_t lmax, int32_t lmin, int32_t dl,
                      int32_t nbins, double* out_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_cl_bin(c, cl_dev, lmax, lmin, dl, nbins, out_dev);
}

ufc_status ufc_alm2map(ufc_ctx* c, const double* alm_dev, int32_t nside, int32_t lmax,
                       float* map_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_alm2map(c, alm_dev, nside, lmax, map_dev);
}

ufc_status ufc_alm_beam(ufc_ctx* c, const double* alm_in_dev, int32_t lmax, double sigma,
                        double* alm_out_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_alm_beam(c, alm_in_dev, lmax, sigma, alm_out_dev);
}

ufc_status ufc_map_stats(ufc_ctx* c, const float* map_dev, int32_t nside, double pdf_lo,
                         double pdf_hi, int32_t nbins, double* moments_dev, int64_t* pdf_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_map_stats(c, map_dev, nside, pdf_lo, pdf_hi, nbins, moments_dev, pdf_dev);
}

ufc_status ufc_bin_host_stream(ufc_ctx* c, const float* const* xyz_host, const int64_t* n,
                               const ufc_box* boxes, int32_t nbox, const double* chi_edges,
                               int32_t nshell, int32_t nside, int32_t flags, int64_t chunk,
                               int32_t* counts_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!xyz_host || !n || !boxes || !chi_edges || !counts_dev)
    return set_err(c, UFC_ERR_ARG, "NULL argument to ufc_bin_host_stream");
  if (flags & ~(UFC_BIN_ACCUMULATE | UFC_BIN_FORCE_DIRECT | UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "unknown flags");
  if ((flags & UFC_BIN_FORCE_DIRECT) && (flags & UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "FORCE_DIRECT and FORCE_DENSE exclude each other");
  if (reinterpret_cast<uintptr_t>(counts_dev) & 3)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 4-byte aligned");
  cudaSetDevice(c->device);
  cudaStreamCaptureStatus cs;
  UFC_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return set_err(c, UFC_ERR_UNSUPPORTED, "ufc_bin_host_stream cannot be captured into a graph");
  return run_bin_stream(c, xyz_host, n, boxes, nbox, chi_edges, nshell, nside, flags, chunk,
                        counts_dev);
}

ufc_status ufc_snapshot_assign(const double* z_edges, int32_t nshell, const double* z_snap,
                               int32_t nsnap, int32_t* snap_of_shell) {
  if (!z_edges || !z_snap || !snap_of_shell || nshell < 1 || nshell > UFC_MAX_SHELLS || nsnap < 1)
    return UFC_ERR_ARG;
  for (int b = 0; b <= nshell; ++b)
    if (!std::isfinite(z_edges[b]) || (b > 0 && !(z_edges[b] > z_edges[b - 1]))) return UFC_ERR_ARG;
  for (int s = 0; s < nsnap; ++s)
    if (!std::isfinite(z_snap[s]) || (s > 0 && !(z_snap[s] > z_snap[s - 1]))) return UFC_ERR_ARG;
  // both lists ascend: one merge pass
  int s = -1;
  for (int b = 0; b < nshell; ++b) {
    const double lim = z_edges[b] + 1e-9 * (1.0 + std::fabs(z_edges[b]));
    while (s + 1 < nsnap && z_snap[s + 1] <= lim) ++s;
    snap_of_shell[b] = s;
  }
  return UFC_OK;
}

}  // extern "C"

// Snapshot-mode binning shared by the device and host-memory entry points:
// argument checks, then the runs of consecutive shells taken from one
// snapshot as boxes owning those shells, kMaxBoxes per pass (the passes
// after the first accumulate).  pass(rx, rn, rb, nrun, flags) bins one pass.
template <class Pass>
static ufc_status bin_snapshot_runs(ufc_ctx* c, const char* who, const float* const* xyz,
                                    const int64_t* n, const ufc_box* snap_geom, int32_t nsnap,
                                    const int32_t* snap_of_shell, const double* chi_edges,
                                    int32_t nshell, int32_t nside, int32_t flags,
                                    int32_t* counts_dev, Pass pass) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!xyz || !n || !snap_geom || !snap_of_shell || !chi_edges || !counts_dev)
    return set_err(c, UFC_ERR_ARG, "NULL argument to %s", who);
  if (nsnap < 1) return set_err(c, UFC_ERR_ARG, "nsnap must be >= 1");
  if (nshell < 1 || nshell > UFC_MAX_SHELLS)
    return set_err(c, UFC_ERR_ARG, "nshell must be in [1,%d]", UFC_MAX_SHELLS);
  if (flags & ~(UFC_BIN_ACCUMULATE | UFC_BIN_FORCE_DIRECT | UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "unknown flags");
  if ((flags & UFC_BIN_FORCE_DIRECT) && (flags & UFC_BIN_FORCE_DENSE))
    return set_err(c, UFC_ERR_ARG, "FORCE_DIRECT and FORCE_DENSE exclude each other");
  if (reinterpret_cast<uintptr_t>(counts_dev) & 3)
    return set_err(c, UFC_ERR_ARG, "counts_dev must be 4-byte aligned");
  for (int b = 0; b < nshell; ++b)
    if (snap_of_shell[b] < -1 || snap_of_shell[b] >= nsnap)
      return set_err(c, UFC_ERR_ARG, "snap_of_shell[%d] = %d outside [-1,%d)", b,
                     snap_of_shell[b], nsnap);
  cudaSetDevice(c->device);
  ufc_box rb[kMaxBoxes];
  const float* rx[kMaxBoxes];
  int64_t rn[kMaxBoxes];
  int nrun = 0, passes = 0;
  auto flush = [&]() -> ufc_status {
    const int32_t f = flags | (passes > 0 ? UFC_BIN_ACCUMULATE : 0);
    const ufc_status st = pass(rx, rn, rb, nrun, f);
    ++passes;
    nrun = 0;
    return st;
  };
  for (int b = 0; b < nshell;) {
    const int s = snap_of_shell[b];
    int e = b + 1;
    while (e < nshell && snap_of_shell[e] == s) ++e;
    if (s >= 0) {
      if (nrun == kMaxBoxes) {
        const ufc_status st = flush();
        if (st) return st;
      }
      rb[nrun] = snap_geom[s];
      rb[nrun].shell_lo = b;
      rb[nrun].shell_hi = e;
      rx[nrun] = xyz[s];
      rn[nrun] = n[s];
      ++nrun;
    }
    b = e;
  }
  if (nrun > 0) return flush();
  if (passes == 0 && !(flags & UFC_BIN_ACCUMULATE))   // no shell has a snapshot
    UFC_CUDA(c, cudaMemsetAsync(counts_dev, 0, (size_t)nshell * 12 * nside * nside * 4, c->stream));
  return UFC_OK;
}

extern "C" {

ufc_status ufc_bin_snapshots(ufc_ctx* c, const float* const* xyz_dev, const int64_t* n,
                             const ufc_box* snap_geom, int32_t nsnap, const int32_t* snap_of_shell,
                             const double* chi_edges, int32_t nshell, int32_t nside, int32_t flags,
                             int32_t* counts_dev) {
  return bin_snapshot_runs(
      c, "ufc_bin_snapshots", xyz_dev, n, snap_geom, nsnap, snap_of_shell, chi_edges, nshell,
      nside, flags, counts_dev,
      [&](const float* const* rx, const int64_t* rn, const ufc_box* rb, int nrun, int32_t f) {
        return run_keys_pipeline(c, 1, rx, rn, rb, nrun, chi_edges, nshell, nside, f, counts_dev,
                                 nullptr, nullptr);
      });
}

ufc_status ufc_bin_snapshots_host(ufc_ctx* c, const float* const* xyz_host, const int64_t* n,
                                  const ufc_box* snap_geom, int32_t nsnap,
                                  const int32_t* snap_of_shell, const double* chi_edges,
                                  int32_t nshell, int32_t nside, int32_t flags, int64_t chunk,
                                  int32_t* counts_dev) {
  if (c) {
    cudaSetDevice(c->device);
    cudaStreamCaptureStatus cs;
    UFC_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return set_err(c, UFC_ERR_UNSUPPORTED, "ufc_bin_snapshots_host cannot be captured into a graph");
  }
  if (chunk < 1) return c ? set_err(c, UFC_ERR_ARG, "chunk must be >= 1") : UFC_ERR_ARG;
  return bin_snapshot_runs(
      c, "ufc_bin_snapshots_host", xyz_host, n, snap_geom, nsnap, snap_of_shell, chi_edges,
      nshell, nside, flags, counts_dev,
      [&](const float* const* rx, const int64_t* rn, const ufc_box* rb, int nrun, int32_t f) {
        return run_bin_stream(c, rx, rn, rb, nrun, chi_edges, nshell, nside, f, chunk,
                              counts_dev);
      });
}

ufc_status ufc_bin_info(ufc_ctx* c, int64_t info[4]) {
  if (!c || !info) return UFC_ERR_ARG;
  BinCounters h;
  cudaSetDevice(c->device);
  UFC_CUDA(c, cudaMemcpyAsync(&h, c->counters, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  UFC_CUDA(c, cudaStreamSynchronize(c->stream));
  info[0] = (int64_t)h.invalid;
  info[1] = (int64_t)h.keyed;
  info[2] = (int64_t)h.refined;
  info[3] = (int64_t)h.exact;
  return UFC_OK;
}

ufc_status ufc_kappa_stats(ufc_ctx* c, const int32_t* counts_dev, int32_t nshell, int32_t nside,
                           const double* A, double C, double pdf_lo, double pdf_hi,
                           int32_t nbins, float* kappa_dev, double* moments_dev,
                           int64_t* pdf_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_kappa_stats(c, counts_dev, nshell, nside, A, C, pdf_lo, pdf_hi, nbins, kappa_dev,
                         moments_dev, pdf_dev);
}

ufc_status ufc_kappa_stats_noalloc(ufc_ctx* c, const int32_t* counts_dev, int32_t nshell,
                                   int32_t nside, const double* A, double C, double pdf_lo,
                                   double pdf_hi, int32_t nbins, float* kappa_dev,
                                   double* moments_dev, int64_t* pdf_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, UFC_ERR_CUDA, "cudaSetDevice(%d) failed", c->device);
  }
  return run_kappa_stats_noalloc(c, counts_dev, nshell, nside, A, C, pdf_lo, pdf_hi, nbins,
                                 kappa_dev, moments_dev, pdf_dev);
}

ufc_status ufc_kappa_backward(ufc_ctx* c, const int32_t* counts_dev, int32_t nshell,
                              int32_t nside, const double* A, double C, double w_var,
                              double w_skew, const float* g_kappa_dev, const double* dA,
                              const double* dC, double* grad_theta, double* G, double* H) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!std::isfinite(w_var) || !std::isfinite(w_skew))
    return set_err(c, UFC_ERR_ARG, "weights must be finite");
  cudaSetDevice(c->device);
  return run_kappa_backward(c, counts_dev, nshell, nside, A, C, w_var, w_skew, g_kappa_dev, dA,
                            dC, grad_theta, G, H);
}

ufc_status ufc_kappa_stats_backward(ufc_ctx* c, const int32_t* counts_dev, int32_t nshell,
                                    int32_t nside, const double* A, double C, double pdf_lo,
                                    double pdf_hi, int32_t nbins, double w_var, double w_skew,
                                    const float* g_kappa_dev, const double* dA, const double* dC,
                                    float* kappa_dev, double* moments_dev, int64_t* pdf_dev,
                                    double* grad_theta, double* G, double* H) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (!std::isfinite(w_var) || !std::isfinite(w_skew))
    return set_err(c, UFC_ERR_ARG, "weights must be finite");
  if (!kappa_dev) return set_err(c, UFC_ERR_ARG, "kappa_dev is NULL");
  cudaSetDevice(c->device);
  return run_kappa_backward_ex(c, counts_dev, nshell, nside, A, C, w_var, w_skew, g_kappa_dev, dA,
                               dC, grad_theta, G, H, kappa_dev, pdf_lo, pdf_hi, nbins, moments_dev,
                               pdf_dev);
}

ufc_status ufc_kappa_partial(ufc_ctx* c, const int32_t* counts_dev, int32_t nshell,
                             int32_t nside, const double* A, double* partial_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_kappa_partial(c, counts_dev, nshell, nside, A, partial_dev);
}

ufc_status ufc_kappa_stats_partial(ufc_ctx* c, const double* partial_dev, int32_t nside,
                                   double C, double pdf_lo, double pdf_hi, int32_t nbins,
                                   float* kappa_dev, double* moments_dev, int64_t* pdf_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_kappa_stats_partial(c, partial_dev, nside, C, pdf_lo, pdf_hi, nbins, kappa_dev,
                                 moments_dev, pdf_dev);
}

ufc_status ufc_kappa_adjoint_sums(ufc_ctx* c, const int32_t* counts_dev, int32_t nshell,
                                  int32_t nside, const double* partial_dev, double C,
                                  const float* g_kappa_dev, double pdf_lo, double pdf_hi,
                                  int32_t nbins, float* kappa_dev, double* moments_dev,
                                  int64_t* pdf_dev, double* sums) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_kappa_adjoint_sums(c, counts_dev, nshell, nside, partial_dev, C, g_kappa_dev,
                                kappa_dev, pdf_lo, pdf_hi, nbins, moments_dev, pdf_dev, sums);
}

ufc_status ufc_kappa_grad_from_sums(const double* sums, int32_t nshell, int32_t nside,
                                    double w_var, double w_skew, const double* dA,
                                    const double* dC, double* grad_theta, double* G, double* H) {
  if (!sums || !dA || !dC || !grad_theta) return UFC_ERR_ARG;
  if (nshell < 1 || nshell > kMaxShells) return UFC_ERR_ARG;
  if (nside < 1 || nside > UFC_MAX_NSIDE || (nside & (nside - 1))) return UFC_ERR_ARG;
  if (!std::isfinite(w_var) || !std::isfinite(w_skew)) return UFC_ERR_ARG;
  for (int k = 0; k < 4 * nshell + 4; ++k)
    if (!std::isfinite(sums[k])) return UFC_ERR_ARG;
  grad_from_sums(sums, nshell, 12 * nside * nside, w_var, w_skew, dA, dC, grad_theta, G, H);
  return UFC_OK;
}

ufc_status ufc_stats_vector(ufc_ctx* c, const double* moments_dev, const int64_t* pdf_dev,
                            int32_t nbins, double* v_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_stats_vector(c, moments_dev, pdf_dev, nbins, v_dev);
}

// Lane k of c (k >= 1) for ufc_batched_stats: a context on c's device with
// its own workspace, counters and stream.
static ufc_ctx* lane_of(ufc_ctx* c, int k) {
  if (!c->lane_stream[k] &&
      cudaStreamCreateWithFlags(&c->lane_stream[k], cudaStreamNonBlocking) != cudaSuccess)
    return nullptr;
  if (!c->lanes[k]) {
    ufc_ctx* l = new (std::nothrow) ufc_ctx();
    if (!l) return nullptr;
    l->device = c->device;
    l->num_sms = c->num_sms;
    l->smem_optin = c->smem_optin;
    l->owner = c;
    if (cudaMalloc(&l->counters, sizeof(BinCounters)) != cudaSuccess) {
      cudaGetLastError();
      delete l;
      return nullptr;
    }
    cudaMemsetAsync(l->counters, 0, sizeof(BinCounters), c->lane_stream[k]);
    c->lanes[k] = l;
  }
  c->lanes[k]->stream = c->lane_stream[k];
  return c->lanes[k];
}

// Count maps up to this size run ufc_batched_stats on concurrent lanes.
constexpr size_t kLaneMapMax = 64ull << 20;

ufc_status ufc_batched_stats(ufc_ctx* c, int32_t nreal, int32_t nbox, const float* const* xyz,
                             const int64_t* n, const ufc_box* boxes, const double* chi,
                             int32_t nshell, int32_t nside, const double* A, const double* C,
                             double lo, double hi, int32_t nbins, int32_t* counts, float* kappa,
                             double* moments, int64_t* pdf, double* stats, double* state,
                             int32_t flags) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  if (nreal < 1 || nbox < 1 || !xyz || !n || !boxes || !chi || !A || !C || !counts || !kappa ||
      !moments || !pdf || !stats || !state)
    return set_err(c, UFC_ERR_ARG, "ufc_batched_stats: bad arguments");
  if (flags & ~(UFC_BATCH_GRAPH | UFC_BATCH_LAUNCHES)) return set_err(c, UFC_ERR_ARG, "unknown flags");
  if (nshell < 1 || nshell > UFC_MAX_SHELLS) return set_err(c, UFC_ERR_ARG, "bad nshell");
  if (nbins < 1 || nbins > 4096) return set_err(c, UFC_ERR_ARG, "bad nbins");
  cudaSetDevice(c->device);
  // grow every workspace slot once for the largest realisation
  int64_t max_img = 0;
  for (int r = 0; r < nreal; ++r) {
    int64_t t = 0;
    for (int k = 0; k < nbox; ++k) {
      const int R = boxes[r * nbox + k].replicate;
      t += n[r * nbox + k] * (int64_t)(2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    }
    max_img = std::max(max_img, t);
  }
  const int d = 6 + nbins;
  const int64_t npix_b = 12ll * nside * nside;
  // one persistent kernel for small maps without periodic images whose maps
  // fit in 4 GB of workspace together
  bool persistent = !(flags & UFC_BATCH_LAUNCHES) && (size_t)nshell * npix_b * 4 <= kLaneMapMax;
  for (int i = 0; i < nreal * nbox && persistent; ++i) persistent = boxes[i].replicate == 0;
  size_t pmaps = 0, pdesc = 0;
  if (persistent) {
    batch_persistent_bytes(c, nreal, nbox, nshell, nside, &pmaps, &pdesc);
    persistent = pmaps <= (4ull << 30);
  }
  char* bmaps = nullptr;
  char* bdesc = nullptr;
  ufc_status s = UFC_OK;
  if (persistent) {
    bmaps = (char*)ws_get(c, kSlotBatchMaps, pmaps);
    bdesc = (char*)ws_get(c, kSlotBatchDesc, pdesc);
    if (!bmaps || !bdesc) return UFC_ERR_ALLOC;
    // descriptors uploaded now, before any capture (also before a cached
    // graph's relaunch, which reads them)
    s = batch_persistent_prepare(c, nreal, nbox, xyz, n, boxes, chi, nshell, nside, A, C, lo, hi,
                                 nbins, moments, pdf, stats, state, bmaps, bdesc);
    if (s) return s;
  } else {
    s = reserve_bin_workspace(c, nbox, max_img, nshell, nside);
    if (s) return s;
    // per-block partial sums of the kappa and moment kernels
    if (!ws_get(c, kSlotPartials, (size_t)16 * c->num_sms * 8)) return UFC_ERR_ALLOC;
  }
  // small maps: realisation r runs on lane r mod nlane, the lanes concurrently
  // (lane 0 is this context with the caller's scratch maps; the others have
  // their own count and kappa maps, workspace and stream)
  const int64_t npix = 12ll * nside * nside;
  const size_t map_bytes = (size_t)nshell * npix * 4;
  // (and a bound of 8 GB on the lanes' binning workspace, ~16 B per image)
  const int64_t ws_lanes = std::max<int64_t>(1, (8ll << 30) / std::max<int64_t>(1, 16 * max_img));
  const int nlane = persistent ? 1
                   : map_bytes <= kLaneMapMax
                        ? (int)std::min<int64_t>({ufc_ctx::kMaxLanes, nreal, ws_lanes})
                        : 1;
  ufc_ctx* lane[ufc_ctx::kMaxLanes] = {c};
  int32_t* lane_counts[ufc_ctx::kMaxLanes] = {counts};
  float* lane_kappa[ufc_ctx::kMaxLanes] = {kappa};
  for (int k = 1; k < nlane; ++k) {
    lane[k] = lane_of(c, k);
    if (!lane[k]) return set_err(c, UFC_ERR_ALLOC, "could not create a batch lane");
    s = reserve_bin_workspace(lane[k], nbox, max_img, nshell, nside);
    if (s) return set_err(c, s, "%s", lane[k]->err.c_str());
    char* m = (char*)ws_get(lane[k], kSlotLaneMap, map_bytes + (size_t)npix * 4 + 256);
    if (!m || !ws_get(lane[k], kSlotPartials, (size_t)16 * c->num_sms * 8))
      return set_err(c, UFC_ERR_ALLOC, "%s", lane[k]->err.c_str());
    lane_counts[k] = reinterpret_cast<int32_t*>(m);
    lane_kappa[k] = reinterpret_cast<float*>(m + ((map_bytes + 255) & ~(size_t)255));
  }
  for (int k = 0; k <= nlane; ++k)
    if (!c->lane_ev[k]) UFC_CUDA(c, cudaEventCreateWithFlags(&c->lane_ev[k], cudaEventDisableTiming));
  const bool graph = (flags & UFC_BATCH_GRAPH) != 0;
  const bool prof = c->prof;
  cudaGraph_t g = nullptr;
  cudaStream_t user = c->stream;
  std::vector<unsigned char> key;
  if (graph) {
    cudaStreamCaptureStatus cs;
    UFC_CUDA(c, cudaStreamIsCapturing(user, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return set_err(c, UFC_ERR_ARG, "the context stream is already capturing");
    if (user == nullptr) {
      // the legacy default stream cannot be captured: capture on the
      // context's own stream, ordered after the work already enqueued
      if (!c->aux_stream)
        UFC_CUDA(c, cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
      for (cudaEvent_t& e : c->aux_ev)
        if (!e) UFC_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      UFC_CUDA(c, cudaEventRecord(c->aux_ev[0], user));
      UFC_CUDA(c, cudaStreamWaitEvent(c->aux_stream, c->aux_ev[0], 0));
    }
    cudaStream_t launch = user ? user : c->aux_stream;
    // the host arguments, byte for byte: an identical call relaunches the
    // cached graph (which re-reads the particle buffers) without capture
    auto put = [&](const void* p, size_t nb) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      key.insert(key.end(), b, b + nb);
    };
    const size_t nrb = (size_t)nreal * nbox;
    put(&nreal, 4); put(&nbox, 4); put(&nshell, 4); put(&nside, 4); put(&nbins, 4);
    const int32_t mode[3] = {persistent ? 1 : 0, c->batch_chunk, c->batch_blocks_per_sm};
    put(mode, sizeof mode);
    put(&lo, 8); put(&hi, 8);
    put(xyz, nrb * sizeof(void*)); put(n, nrb * 8);
    for (size_t i = 0; i < nrb; ++i) {
      const ufc_box& b = boxes[i];
      put(&b.L, 8); put(b.obs, 24); put(&b.n_total, 8);
      put(&b.shell_lo, 4); put(&b.shell_hi, 4); put(&b.replicate, 4);
    }
    put(chi, (size_t)(nshell + 1) * 8); put(A, (size_t)nreal * nshell * 8); put(C, (size_t)nreal * 8);
    const void* outs[6] = {counts, kappa, moments, pdf, stats, state};
    put(outs, sizeof outs);
    if (c->graph_exec && key == c->graph_key) {
      UFC_CUDA(c, cudaGraphLaunch(c->graph_exec, launch));
      if (launch != user) {
        UFC_CUDA(c, cudaEventRecord(c->aux_ev[1], launch));
        UFC_CUDA(c, cudaStreamWaitEvent(user, c->aux_ev[1], 0));
      }
      return UFC_OK;
    }
    c->stream = launch;
    c->prof = false;   // event records would become graph nodes
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      c->stream = user;
      c->prof = prof;
      return set_err(c, UFC_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
  }
  // fork: the lanes start after the work already on this context's stream
  if (nlane > 1) {
    UFC_CUDA(c, cudaEventRecord(c->lane_ev[0], c->stream));
    for (int k = 1; k < nlane; ++k) UFC_CUDA(c, cudaStreamWaitEvent(lane[k]->stream, c->lane_ev[0], 0));
  }
  if (persistent) s = batch_persistent_enqueue(c, bmaps, bdesc);
  for (int r = 0; r < nreal && !s && !persistent; ++r) {
    ufc_ctx* lc = lane[r % nlane];
    int32_t* cnt = lane_counts[r % nlane];
    float* kap = lane_kappa[r % nlane];
    s = run_keys_pipeline(lc, 1, xyz + r * nbox, n + r * nbox, boxes + r * nbox, nbox, chi, nshell,
                          nside, 0, cnt, nullptr, nullptr);
    if (!s)
      s = run_kappa_stats(lc, cnt, nshell, nside, A + (size_t)r * nshell, C[r], lo, hi, nbins,
                          kap, moments + 10 * (size_t)r, pdf + (size_t)(nbins + 3) * r);
    if (!s) s = run_stats_vector(lc, moments + 10 * (size_t)r, pdf + (size_t)(nbins + 3) * r, nbins,
                                 stats + (size_t)d * r);
    if (s && lc != c) set_err(c, s, "%s", lc->err.c_str());
  }
  // join: the Welford update (in realisation order) waits for every lane
  for (int k = 1; k < nlane; ++k) {
    const cudaError_t e = cudaEventRecord(c->lane_ev[k], lane[k]->stream);
    if (e == cudaSuccess) cudaStreamWaitEvent(c->stream, c->lane_ev[k], 0);
    else if (!s) s = set_err(c, UFC_ERR_CUDA, "lane join: %s", cudaGetErrorString(e));
  }
  if (!s && !persistent) s = run_welford_update(c, stats, nreal, d, state);
  if (graph) {
    cudaStream_t cap = c->stream;
    c->stream = user;
    c->prof = prof;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (s) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return set_err(c, UFC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    // reuse the cached executable graph when only parameters changed
    bool updated = false;
    if (c->graph_exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(c->graph_exec, g, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
      }
    }
    if (!updated) e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) {
      c->graph_key.swap(key);
      e = cudaGraphLaunch(c->graph_exec, cap);
    } else {
      c->graph_exec = nullptr;
      c->graph_key.clear();
    }
    if (e == cudaSuccess && cap != user) {      // join: later work on the caller's stream waits
      e = cudaEventRecord(c->aux_ev[1], cap);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(user, c->aux_ev[1], 0);
    }
    if (e != cudaSuccess) return set_err(c, UFC_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(e));
  }
  return s;
}

ufc_status ufc_welford_update(ufc_ctx* c, const double* v_dev, int32_t nvec, int32_t d,
                              double* state_dev) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_welford_update(c, v_dev, nvec, d, state_dev);
}

ufc_status ufc_welford_merge(ufc_ctx* c, double* a, const double* b, int32_t d) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_welford_merge(c, a, b, d);
}

ufc_status ufc_welford_finalize(ufc_ctx* c, const double* st, int32_t d, int32_t ddof,
                                double* mean, double* cov, double* corr) {
  if (!c) return UFC_ERR_ARG;
  c->err.clear();
  cudaSetDevice(c->device);
  return run_welford_finalize(c, st, d, ddof, mean, cov, corr);
}

}  // extern "C"
