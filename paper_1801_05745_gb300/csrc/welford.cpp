// Welford update and Chan merge of covariance states on host memory (Eq. 10,
// the realisation-sharded path): the same formulas, in the same order, as
// k_welford_update and k_welford_merge of the device library.
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/ufalcon.h"

extern "C" ufc_status ufc_welford_update_host(const double* v, int32_t nvec, int32_t d,
                                              double* st) {
  if (!v || !st || nvec < 0 || d < 1 || d > 8192) return UFC_ERR_ARG;
  double* mean = st + 1;
  double* M2 = st + 1 + d;
  std::vector<double> dold(d), dnew(d);
  const double n0 = st[0];
  for (int32_t r = 0; r < nvec; ++r) {
    const double* x = v + (size_t)r * d;
    const double n = n0 + double(r + 1);
    for (int32_t i = 0; i < d; ++i) {
      const double delta = x[i] - mean[i];
      const double mn = mean[i] + delta / n;
      dold[i] = delta;
      dnew[i] = x[i] - mn;
    }
    for (int32_t i = 0; i < d; ++i)
      for (int32_t j = 0; j < d; ++j) M2[(size_t)i * d + j] += dold[i] * dnew[j];
    for (int32_t i = 0; i < d; ++i) mean[i] += dold[i] / n;
  }
  st[0] = n0 + double(nvec);
  return UFC_OK;
}

extern "C" ufc_status ufc_welford_merge_host(double* a, const double* b, int32_t d) {
  if (!a || !b || d < 1 || d > 8192) return UFC_ERR_ARG;
  const double na = a[0], nb = b[0], n = na + nb;
  if (nb == 0.0) return UFC_OK;
  double* ma = a + 1;
  const double* mb = b + 1;
  double* Ma = a + 1 + d;
  const double* Mb = b + 1 + d;
  const double f = (n > 0.0) ? na * nb / n : 0.0;
  for (int32_t i = 0; i < d; ++i)
    for (int32_t j = 0; j < d; ++j) {
      const size_t k = (size_t)i * d + j;
      Ma[k] += Mb[k] + (mb[i] - ma[i]) * (mb[j] - ma[j]) * f;
    }
  for (int32_t i = 0; i < d; ++i) ma[i] += (mb[i] - ma[i]) * nb / n;
  a[0] = n;
  return UFC_OK;
}
