// Batched searches (trstmi_batch_*, include/trstmi.h): many independent
// instances of different (N, d) advanced together, each iteration one set of
// shared launches for all of them, replayed from a captured CUDA graph.
//
// Every instance keeps its own device state, seed and counters, and a pair's
// |G|^2 is computed by the same sequential chain whatever the tile width, so
// an instance follows exactly the trajectory it follows alone.
//
// Tile widths: the scoring kernel is instantiated for tiles of 16, 32 and 64
// columns.  The autotuner times the persistent scoring pass on the actual
// instances of each (d, ceil log2 N) bucket at every feasible width and
// keeps the fastest; the choice is cached for the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/trstmi.h"
#include "kernels.h"

using namespace trstmi;

namespace {

constexpr int kBatchGraphChunk = 16;

__global__ void k_batch_set_stop(SlotDesc* slots, int n, uint32_t iters) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  DevState* st = slots[s].st;
  const unsigned long long stop = (unsigned long long)st->t + iters;
  st->t_stop = stop > 0xffffffffull ? 0xffffffffu : (uint32_t)stop;
  st->t_call = st->t;
  st->accepts_call = st->accepts;
}

template <typename B>
__global__ void k_batch_set_mu2cur(SlotDesc* slots, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  DevState* st = slots[s].st;
  st->mu2_cur = (double)nonneg_from_bits(reinterpret_cast<const B*>(slots[s].mu2)[0]);
  st->done = (st->mu2_cur <= st->target2) ? 1u : 0u;
}

std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned_R[2];   // [f64] (d, ceil log2 N) -> R

int ceil_log2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

int ntiles_for(int N, int R) {
  const int nb = (N + 16 * R - 1) / (16 * R);
  return nb * (nb + 1) / 2;
}

}  // namespace

namespace trstmi {
// Width cache shared with the serving loop.
int cached_width(bool f64, int d, int N) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned_R[f64].find({d, ceil_log2(N)});
  return it == g_tuned_R[f64].end() ? 0 : it->second;
}
void store_width(bool f64, int d, int N, int R) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned_R[f64][{d, ceil_log2(N)}] = R;
}
int tiles_at_width(int N, int R) { return ntiles_for(N, R); }
}  // namespace trstmi

struct trstmi_batch {
  int n = 0;
  trstmi_options opt{};
  bool f64 = false;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* block = nullptr;
  std::vector<int> N, d;
  std::vector<uint64_t> seed;
  std::vector<SlotDesc> h_slots;
  SlotDesc* d_slots = nullptr;
  int maxN = 0;
  struct Group {
    int R = 1;
    int* d_ids = nullptr;
    long long* d_begin = nullptr;
    int count = 0;
    long long nitems = 0;
    size_t smem = 0;
    int grid = 0;
  };
  std::vector<Group> groups;
  unsigned long long* d_counters = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<void*> extra;   // group tables (cudaMalloc'd)
};

namespace {

#define BTRY(expr)                                     \
  do {                                                 \
    if ((expr) != cudaSuccess) { cudaGetLastError(); return TRSTMI_ECUDA; } \
  } while (0)

int build_group(trstmi_batch* b, int R, std::vector<int> ids, trstmi_batch::Group* g) {
  // heaviest instances first: their items are handed out first
  auto cost = [&](int i) {
    return (double)b->h_slots[i].K * ntiles_for(b->N[i], R) * (16.0 * R) * (16.0 * R) * b->d[i];
  };
  std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::vector<long long> begin(ids.size() + 1, 0);
  size_t smem = 0;
  for (size_t q = 0; q < ids.size(); ++q) {
    const int i = ids[q];
    const long long items = (long long)b->h_slots[i].K * ntiles_for(b->N[i], R);
    begin[q + 1] = begin[q] + items;
    smem = std::max(smem, gram_smem_bytes(b->f64, b->d[i], R));
  }
  g->R = R;
  g->count = (int)ids.size();
  g->nitems = begin.back();
  g->smem = smem;
  int per_sm = 0;
  BTRY(batch_score_occupancy(b->f64, R, smem, &per_sm));
  if (per_sm < 1) return TRSTMI_EUNSUPPORTED;
  g->grid = (int)std::min<long long>(g->nitems, (long long)b->num_sms * per_sm);
  BTRY(cudaMalloc(&g->d_ids, sizeof(int) * std::max<size_t>(ids.size(), 1)));
  BTRY(cudaMalloc(&g->d_begin, sizeof(long long) * begin.size()));
  b->extra.push_back(g->d_ids);
  b->extra.push_back(g->d_begin);
  BTRY(cudaMemcpy(g->d_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(g->d_begin, begin.data(), sizeof(long long) * begin.size(),
                  cudaMemcpyHostToDevice));
  return TRSTMI_OK;
}

bool width_feasible(bool f64, int d, int N, int R) {
  if (gram_smem_bytes(f64, d, R) > 200 * 1024) return false;
  return R == 1 || 16 * R < 2 * N;     // do not pad tiny N
}

int apply_widths(trstmi_batch* b, const std::vector<int>& R_of) {
  for (int i = 0; i < b->n; ++i) {
    b->h_slots[i].R = R_of[i];
    b->h_slots[i].ntiles = ntiles_for(b->N[i], R_of[i]);
  }
  b->groups.clear();
  for (int R : {4, 2, 1}) {
    std::vector<int> ids;
    for (int i = 0; i < b->n; ++i)
      if (R_of[i] == R) ids.push_back(i);
    if (ids.empty()) continue;
    trstmi_batch::Group g;
    int rc = build_group(b, R, ids, &g);
    if (rc) return rc;
    b->groups.push_back(g);
  }
  BTRY(cudaMemcpy(b->d_slots, b->h_slots.data(), sizeof(SlotDesc) * b->n, cudaMemcpyHostToDevice));
  return TRSTMI_OK;
}

// Times one scoring pass of the given instances at width R (ms, CUDA events).
int time_width(trstmi_batch* b, const std::vector<int>& ids, int R, float* ms) {
  // the descriptors must carry this width while it is timed
  std::vector<SlotDesc> saved = b->h_slots;
  for (int i : ids) { b->h_slots[i].R = R; b->h_slots[i].ntiles = ntiles_for(b->N[i], R); }
  BTRY(cudaMemcpy(b->d_slots, b->h_slots.data(), sizeof(SlotDesc) * b->n, cudaMemcpyHostToDevice));
  trstmi_batch::Group g;
  int rc = build_group(b, R, ids, &g);
  if (rc) { b->h_slots = saved; return rc; }
  cudaStream_t s = b->stream;
  float best = 1e30f;
  for (int rep = 0; rep < 3 && rc == TRSTMI_OK; ++rep) {
    if (cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long), s) != cudaSuccess ||
        cudaEventRecord(b->ev0, s) != cudaSuccess ||
        launch_batch_score(b->f64, R, b->d_slots, g.d_ids, g.d_begin, g.count, g.nitems,
                           b->d_counters, g.smem, g.grid, s) != cudaSuccess ||
        cudaEventRecord(b->ev1, s) != cudaSuccess || cudaEventSynchronize(b->ev1) != cudaSuccess) {
      rc = TRSTMI_ECUDA;
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, b->ev0, b->ev1);
    if (rep > 0) best = std::min(best, t);   // first launch warms up
  }
  b->h_slots = saved;
  *ms = best;
  return rc;
}

// Chooses every instance's tile width: cached per (d, ceil log2 N), measured
// on the instances of a bucket when it is first seen.
int autotune(trstmi_batch* b) {
  std::map<std::pair<int, int>, std::vector<int>> buckets;
  for (int i = 0; i < b->n; ++i) buckets[{b->d[i], ceil_log2(b->N[i])}].push_back(i);
  std::vector<int> R_of(b->n, 1);
  // instances must be active (and not advance) while widths are timed
  k_batch_set_stop<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_slots, b->n, 1u);
  BTRY(cudaGetLastError());
  BTRY(launch_batch_begin(b->d_slots, b->n, b->d_counters, 1, b->f64, b->stream));
  for (auto& kv : buckets) {
    int R = -1;
    {
      std::lock_guard<std::mutex> g(g_tune_mu);
      auto it = g_tuned_R[b->f64].find(kv.first);
      if (it != g_tuned_R[b->f64].end()) R = it->second;
    }
    if (R < 0) {
      float best = 1e30f;
      for (int cand : {1, 2, 4}) {
        bool ok = true;
        for (int i : kv.second) ok = ok && width_feasible(b->f64, b->d[i], b->N[i], cand);
        if (!ok) continue;
        float ms = 0.f;
        int rc = time_width(b, kv.second, cand, &ms);
        if (rc) return rc;
        if (ms < best) { best = ms; R = cand; }
      }
      if (R < 0) R = 1;
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned_R[b->f64][kv.first] = R;
    }
    for (int i : kv.second) R_of[i] = R;
  }
  return apply_widths(b, R_of);
}

int enqueue_batch_iteration(trstmi_batch* b, cudaStream_t s) {
  BTRY(launch_batch_begin(b->d_slots, b->n, b->d_counters, (int)b->groups.size(), b->f64, s));
  for (size_t g = 0; g < b->groups.size(); ++g) {
    const auto& G = b->groups[g];
    BTRY(launch_batch_score(b->f64, G.R, b->d_slots, G.d_ids, G.d_begin, G.count, G.nitems,
                            b->d_counters + g, G.smem, G.grid, s));
  }
  BTRY(launch_batch_decide(b->d_slots, b->n, b->f64, s));
  BTRY(launch_batch_commit(b->d_slots, b->n, b->maxN, b->f64, s));
  return TRSTMI_OK;
}

int batch_graph(trstmi_batch* b, int iters, cudaGraphExec_t* out) {
  auto it = b->graphs.find(iters);
  if (it != b->graphs.end()) { *out = it->second; return TRSTMI_OK; }
  cudaGraph_t g = nullptr;
  BTRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = TRSTMI_OK;
  for (int i = 0; i < iters && rc == TRSTMI_OK; ++i) rc = enqueue_batch_iteration(b, b->stream);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : TRSTMI_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return TRSTMI_ECUDA;
  b->graphs[iters] = ex;
  *out = ex;
  return TRSTMI_OK;
}

int read_states(trstmi_batch* b, std::vector<DevState>* out) {
  out->resize(b->n);
  for (int i = 0; i < b->n; ++i)
    BTRY(cudaMemcpyAsync(&(*out)[i], b->h_slots[i].st, sizeof(DevState), cudaMemcpyDeviceToHost,
                         b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  return TRSTMI_OK;
}

}  // namespace

extern "C" {

void trstmi_batch_destroy(trstmi_batch_handle b) {
  if (!b) return;
  cudaSetDevice(b->opt.device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (void* p : b->extra) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->block) cudaFree(b->block);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int trstmi_batch_create(int n, const int* N, const int* d, const uint64_t* seeds,
                        const trstmi_options* opt, trstmi_batch_handle* out) {
  if (!out) return TRSTMI_EINVAL;
  *out = nullptr;
  if (n < 1 || !N || !d || !seeds) return TRSTMI_EINVAL;
  trstmi_options o;
  if (opt) o = *opt; else trstmi_default_options(&o);
  if (o.precision != TRSTMI_FP32 && o.precision != TRSTMI_FP64) return TRSTMI_EUNSUPPORTED;
  if (o.K < 1 || o.trace_cap < 0 || !(o.delta0 > 0) || !(o.gamma_inc >= 1) ||
      !(o.gamma_dec > 0 && o.gamma_dec <= 1) || !(o.delta_min >= 0) || !(o.delta_max >= o.delta_min))
    return TRSTMI_EINVAL;
  for (int i = 0; i < n; ++i)
    if (N[i] < 2 || d[i] < 1 || d[i] > kMaxD || (long long)N[i] * ((d[i] + 1) / 2) >= (1ll << 32))
      return TRSTMI_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return TRSTMI_ECUDA;
  if (o.device < 0 || o.device >= ndev) return TRSTMI_EINVAL;
  if (cudaSetDevice(o.device) != cudaSuccess) return TRSTMI_ECUDA;
  if (init_kernel_attributes() != cudaSuccess) return TRSTMI_ECUDA;

  trstmi_batch* b = new (std::nothrow) trstmi_batch();
  if (!b) return TRSTMI_ENOMEM;
  b->n = n; b->opt = o; b->f64 = (o.precision == TRSTMI_FP64);
  b->N.assign(N, N + n); b->d.assign(d, d + n); b->seed.assign(seeds, seeds + n);
  if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess) {
    delete b;
    return TRSTMI_ECUDA;
  }
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return TRSTMI_ECUDA;
    }
    b->own_stream = true;
  }
  // one arena: states, descriptors, counters, then per instance frames, scores, trace
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t K = (size_t)o.K, tcap = (size_t)std::max(o.trace_cap, 1);
  size_t off = 0;
  const size_t o_st = off; off = up(off + sizeof(DevState) * n);
  const size_t o_sl = off; off = up(off + sizeof(SlotDesc) * n);
  const size_t o_ct = off; off = up(off + sizeof(unsigned long long) * 8);
  std::vector<size_t> o_phi64(n), o_phi32(n), o_mu2(n), o_tr(n);
  for (int i = 0; i < n; ++i) {
    const size_t nd = (size_t)N[i] * d[i];
    o_phi64[i] = off; off = up(off + nd * sizeof(double2));
    o_phi32[i] = off; off = up(off + nd * sizeof(float2));
    o_mu2[i] = off; off = up(off + K * sizeof(unsigned long long));
    o_tr[i] = off; off = up(off + tcap * sizeof(TraceRowDev));
    b->maxN = std::max(b->maxN, N[i]);
  }
  if (cudaMalloc(&b->block, off) != cudaSuccess) {
    cudaGetLastError();
    trstmi_batch_destroy(b);
    return TRSTMI_ENOMEM;
  }
  char* base = (char*)b->block;
  DevState* states = (DevState*)(base + o_st);
  b->d_slots = (SlotDesc*)(base + o_sl);
  b->d_counters = (unsigned long long*)(base + o_ct);
  b->h_slots.resize(n);
  std::vector<DevState> s0(n);
  for (int i = 0; i < n; ++i) {
    SlotDesc& sd = b->h_slots[i];
    sd.st = states + i;
    double2* p64 = (double2*)(base + o_phi64[i]);
    float2* p32 = (float2*)(base + o_phi32[i]);
    sd.phi = b->f64 ? (void*)p64 : (void*)p32;
    sd.phi_other = b->f64 ? (void*)p32 : (void*)p64;
    sd.mu2 = base + o_mu2[i];
    sd.trace = (TraceRowDev*)(base + o_tr[i]);
    sd.seed = seeds[i];
    sd.N = N[i]; sd.d = d[i]; sd.K = o.K; sd.R = 1; sd.ntiles = ntiles_for(N[i], 1); sd.pad = 0;
    sd.item_begin = 0;
    DevState& s = s0[i];
    std::memset(&s, 0, sizeof(s));
    s.delta = o.delta0; s.delta_used = o.delta0;
    s.target2 = o.target_mu > 0 ? o.target_mu * o.target_mu : -1.0;
    s.gamma_inc = o.gamma_inc; s.gamma_dec = o.gamma_dec;
    s.delta_min = o.delta_min; s.delta_max = o.delta_max;
    s.screen_min_delta = o.screen_min_delta;
    s.trace_cap = (uint32_t)o.trace_cap;
  }
  cudaStream_t s = b->stream;
  int rc = TRSTMI_OK;
  if (cudaMemsetAsync(b->block, 0, off, s) != cudaSuccess ||
      cudaMemcpyAsync(states, s0.data(), sizeof(DevState) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_slots, b->h_slots.data(), sizeof(SlotDesc) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
    rc = TRSTMI_ECUDA;
  // seeded initial frames and their scores in the deciding precision
  for (int i = 0; i < n && rc == TRSTMI_OK; ++i) {
    SlotDesc& sd = b->h_slots[i];
    double2* p64 = (double2*)(base + o_phi64[i]);
    float2* p32 = (float2*)(base + o_phi32[i]);
    if (launch_init_frame(N[i], d[i], seeds[i], p64, p32, sd.st, s) != cudaSuccess) rc = TRSTMI_ECUDA;
    GramSource src{};
    src.perturb = false;
    src.phi = sd.phi;
    cudaError_t e = b->f64
        ? launch_gram_f64(N[i], d[i], 1, src, (unsigned long long*)sd.mu2, b->num_sms, s)
        : launch_gram_f32(N[i], d[i], 1, src, (unsigned int*)sd.mu2, nullptr, b->num_sms, s);
    if (e != cudaSuccess) rc = TRSTMI_ECUDA;
  }
  if (rc == TRSTMI_OK) {
    if (b->f64) k_batch_set_mu2cur<unsigned long long><<<(n + 127) / 128, 128, 0, s>>>(b->d_slots, n);
    else k_batch_set_mu2cur<unsigned int><<<(n + 127) / 128, 128, 0, s>>>(b->d_slots, n);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = TRSTMI_ECUDA;
  }
  if (rc == TRSTMI_OK) rc = autotune(b);
  if (rc == TRSTMI_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = TRSTMI_ECUDA;
  if (rc == TRSTMI_OK) {
    std::vector<DevState> chk;
    rc = read_states(b, &chk);
    for (int i = 0; rc == TRSTMI_OK && i < n; ++i)
      if (chk[i].error & kErrZeroColumn) rc = TRSTMI_EINVAL;
  }
  if (rc) { trstmi_batch_destroy(b); return rc; }
  *out = b;
  return TRSTMI_OK;
}

int trstmi_batch_step(trstmi_batch_handle b, int iters, trstmi_step_info* info) {
  if (!b || iters < 0) return TRSTMI_EINVAL;
  BTRY(cudaSetDevice(b->opt.device));
  cudaStream_t s = b->stream;
  const int full = iters / kBatchGraphChunk, rem = iters % kBatchGraphChunk;
  cudaGraphExec_t gf = nullptr, gr = nullptr;
  int rc;
  if (full > 0 && (rc = batch_graph(b, kBatchGraphChunk, &gf)) != TRSTMI_OK) return rc;
  if (rem > 0 && (rc = batch_graph(b, rem, &gr)) != TRSTMI_OK) return rc;
  BTRY(cudaEventRecord(b->ev0, s));
  k_batch_set_stop<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_slots, b->n, (uint32_t)iters);
  BTRY(cudaGetLastError());
  for (int r = 0; r < full; ++r) BTRY(cudaGraphLaunch(gf, s));
  if (gr) BTRY(cudaGraphLaunch(gr, s));
  BTRY(cudaEventRecord(b->ev1, s));
  std::vector<DevState> st;
  rc = read_states(b, &st);
  if (rc) return rc;
  uint32_t err = 0;
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    std::memset(info, 0, sizeof(*info));
    int all_done = 1;
    double mu_max = 0.0;
    for (int i = 0; i < b->n; ++i) {
      const int it = (int)(st[i].t - st[i].t_call);
      info->iters_done = std::max(info->iters_done, it);
      info->accepts += (int32_t)(st[i].accepts - st[i].accepts_call);
      info->pairs_scored += (uint64_t)it * (uint64_t)b->opt.K *
                            ((uint64_t)b->N[i] * (uint64_t)(b->N[i] - 1) / 2);
      mu_max = std::max(mu_max, std::sqrt(st[i].mu2_cur));
      all_done &= (int)st[i].done;
    }
    info->mu = mu_max;
    info->delta = 0.0;
    info->elapsed_ns = (uint64_t)((double)ms * 1e6);
    info->done = all_done;
  }
  for (int i = 0; i < b->n; ++i) err |= st[i].error;
  if (err & kErrTimeout) return TRSTMI_ETIMEOUT;
  if (err & kErrZeroColumn) return TRSTMI_EINVAL;
  return TRSTMI_OK;
}

int trstmi_batch_mu(trstmi_batch_handle b, double* mu, int32_t* iters) {
  if (!b || !mu) return TRSTMI_EINVAL;
  BTRY(cudaSetDevice(b->opt.device));
  std::vector<DevState> st;
  int rc = read_states(b, &st);
  if (rc) return rc;
  for (int i = 0; i < b->n; ++i) {
    mu[i] = std::sqrt(st[i].mu2_cur);
    if (iters) iters[i] = (int32_t)st[i].t;
  }
  return TRSTMI_OK;
}

int trstmi_batch_get_phi(trstmi_batch_handle b, int i, double* out) {
  if (!b || !out || i < 0 || i >= b->n) return TRSTMI_EINVAL;
  BTRY(cudaSetDevice(b->opt.device));
  const SlotDesc& sd = b->h_slots[i];
  const void* p64 = b->f64 ? sd.phi : sd.phi_other;
  BTRY(cudaMemcpyAsync(out, p64, (size_t)sd.N * sd.d * sizeof(double2), cudaMemcpyDeviceToHost,
                       b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  return TRSTMI_OK;
}

int trstmi_batch_get_trace(trstmi_batch_handle b, int i, trstmi_trace_row* rows, int n,
                           int* n_out) {
  if (!b || i < 0 || i >= b->n || n < 0 || !n_out || (n > 0 && !rows)) return TRSTMI_EINVAL;
  BTRY(cudaSetDevice(b->opt.device));
  DevState s;
  BTRY(cudaMemcpyAsync(&s, b->h_slots[i].st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
  const uint32_t cap = (uint32_t)b->opt.trace_cap;
  std::vector<TraceRowDev> all(cap ? cap : 1);
  if (cap)
    BTRY(cudaMemcpyAsync(all.data(), b->h_slots[i].trace, cap * sizeof(TraceRowDev),
                         cudaMemcpyDeviceToHost, b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  const uint32_t cnt = std::min<uint32_t>(std::min<uint32_t>(cap, s.t), (uint32_t)n);
  for (uint32_t q = 0; q < cnt; ++q) {
    const uint32_t t = s.t - cnt + 1 + q;
    std::memcpy(&rows[q], &all[(t - 1) % cap], sizeof(TraceRowDev));
  }
  *n_out = (int)cnt;
  return TRSTMI_OK;
}

int trstmi_batch_profile_score(trstmi_batch_handle b, int launches, size_t flush_bytes,
                               double* avg_ms) {
  if (!b || launches < 1 || !avg_ms) return TRSTMI_EINVAL;
  BTRY(cudaSetDevice(b->opt.device));
  cudaStream_t s = b->stream;
  void* flush = nullptr;
  if (flush_bytes) BTRY(cudaMalloc(&flush, flush_bytes));
  double total = 0.0;
  int rc = TRSTMI_OK;
  for (int l = 0; l < launches && rc == TRSTMI_OK; ++l) {
    // make every instance active for one iteration without advancing it
    k_batch_set_stop<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_slots, b->n, 1u);
    if (cudaGetLastError() != cudaSuccess ||
        launch_batch_begin(b->d_slots, b->n, b->d_counters, (int)b->groups.size(), b->f64, s) ||
        (flush && cudaMemsetAsync(flush, l & 0xff, flush_bytes, s)) ||
        cudaEventRecord(b->ev0, s) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    for (size_t g = 0; g < b->groups.size(); ++g) {
      const auto& G = b->groups[g];
      if (launch_batch_score(b->f64, G.R, b->d_slots, G.d_ids, G.d_begin, G.count, G.nitems,
                             b->d_counters + g, G.smem, G.grid, s) != cudaSuccess) rc = TRSTMI_ECUDA;
    }
    float ms = 0.f;
    if (rc || cudaEventRecord(b->ev1, s) != cudaSuccess || cudaEventSynchronize(b->ev1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, b->ev0, b->ev1) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    total += ms;
  }
  if (flush) cudaFree(flush);
  if (rc == TRSTMI_OK) *avg_ms = total / launches;
  return rc;
}

int trstmi_batch_tile_widths(trstmi_batch_handle b, int* widths) {
  if (!b || !widths) return TRSTMI_EINVAL;
  for (int i = 0; i < b->n; ++i) widths[i] = 16 * b->h_slots[i].R;
  return TRSTMI_OK;
}

}  // extern "C"
