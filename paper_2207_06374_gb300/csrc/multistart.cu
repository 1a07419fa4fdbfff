// Multi-start: L random initialisations searched as batched instances and the
// minimum over the trials (arXiv 2207.06374, Algorithm "TRSTMI optimization
// steps", last step; the Remark on the experiments uses L = 2 d^2).  Host
// code over the batch interface: each trial is the search trstmi_create +
// trstmi_step would run alone with its seed, so the result does not depend on
// how the trials are grouped into batches.
#include <algorithm>
#include <vector>

#include "../../include/trstmi.h"
#include "trace.h"

extern "C" int trstmi_multistart(int N, int d, uint64_t seed0, int L, int iters,
                                 const trstmi_options* opt, int batch_cap,
                                 trstmi_multistart_result* out, double* mu_all,
                                 double* best_phi) {
  trstmi::TraceRange trace_range("trstmi_multistart");
  if (!out || N < 2 || d < 1 || iters < 0) return TRSTMI_EINVAL;
  if (L <= 0) L = 2 * d * d;
  const int cap = batch_cap > 0 ? std::min(batch_cap, L) : L;
  std::vector<double> mu(L);
  for (int b0 = 0; b0 < L; b0 += cap) {
    const int n = std::min(cap, L - b0);
    std::vector<int> Ns(n, N), ds(n, d);
    std::vector<uint64_t> seeds(n);
    for (int i = 0; i < n; ++i) seeds[i] = seed0 + (uint64_t)(b0 + i);
    trstmi_batch_handle b = nullptr;
    int rc = trstmi_batch_create(n, Ns.data(), ds.data(), seeds.data(), opt, &b);
    if (rc) return rc;
    if (iters > 0) rc = trstmi_batch_step(b, iters, nullptr);
    if (!rc) rc = trstmi_batch_mu(b, mu.data() + b0, nullptr);
    trstmi_batch_destroy(b);
    if (rc) return rc;
  }
  int best = 0;
  for (int i = 1; i < L; ++i)
    if (mu[i] < mu[best]) best = i;   // lowest index on ties
  out->mu = mu[best];
  out->best = best;
  out->trials = L;
  out->best_seed = seed0 + (uint64_t)best;
  if (mu_all) std::copy(mu.begin(), mu.end(), mu_all);
  if (best_phi) {
    // the winning trial again, alone: the same trajectory, so the same frame
    trstmi_handle h = nullptr;
    int rc = trstmi_create(N, d, out->best_seed, opt, &h);
    if (rc) return rc;
    if (iters > 0) rc = trstmi_step(h, iters, nullptr);
    if (!rc) rc = trstmi_get_phi(h, best_phi);
    trstmi_destroy(h);
    if (rc) return rc;
  }
  return TRSTMI_OK;
}
