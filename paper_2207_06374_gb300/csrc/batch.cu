// Batched searches (trstmi_batch_*, include/trstmi.h): many independent
// instances of different (N, d) advanced together, each iteration one set of
// shared launches for all of them (BatchPlan), replayed from a captured CUDA
// graph.
//
// Every instance keeps its own device state, seed and counters, and a pair's
// |G|^2 is computed by the same sequential chain whatever the tile width, so
// an instance follows exactly the trajectory it follows alone (the screen
// scores one candidate per CTA in either form, so the same holds there).
//
// Tile widths: the fp32/fp64 scoring kernel is instantiated for tiles of 16,
// 32 and 64 columns, and small instances can instead be scored whole (the
// candidate drawn once into shared memory, kResident).  The autotuner times
// the persistent scoring pass on the actual instances of each (d, ceil log2 N)
// bucket at every feasible choice and keeps the fastest; the choice is cached
// for the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/trstmi.h"
#include "kernels.h"
#include "trace.h"

using namespace trstmi;

namespace {

constexpr int kBatchGraphChunk = 16;
constexpr size_t kBatchPlanesMax = 512ull << 20;
// Pair list of the certification: the standalone instance's 65536 pairs, or
// every pair when there are fewer, so that the list overflows exactly when a
// standalone run's does.
uint32_t slot_pair_cap(int N) {
  const unsigned long long all = (unsigned long long)N * (unsigned long long)(N - 1) / 2;
  return (uint32_t)std::min<unsigned long long>(all, 1ull << 16);
}

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

// Screen modes: the initial frame is certified in binary64 like every later
// one, by the certification passes (cert64 of the slot).
__global__ void k_batch_set_mu2cur_cert(SlotDesc* slots, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  DevState* st = slots[s].st;
  st->mu2_cur = nonneg_from_bits(*slots[s].cert64);
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

bool is_screen_prec(int p) { return is_screen_precision(p); }

}  // namespace

namespace trstmi {
// Width cache shared with the serving loop.
int cached_width(bool f64, int d, int N) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned_R[f64].find({d, ceil_log2(N)});
  return it == g_tuned_R[f64].end() ? -1 : it->second;
}
void store_width(bool f64, int d, int N, int R) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned_R[f64][{d, ceil_log2(N)}] = R;
}
int tiles_at_width(int N, int R) { return R == kResident ? 1 : ntiles_for(N, R); }

bool width_feasible(bool f64, int d, int N, int R) {
  // whole candidates up to 48 KiB of shared memory (four CTAs per SM or more)
  if (R == kResident) return resident_smem_bytes(f64, d, N) <= 48 * 1024;
  if (gram_smem_bytes(f64, d, R) > 200 * 1024) return false;
  return R == 1 || 16 * R < 2 * N;     // do not pad tiny N
}

// Times one full scoring pass of the given instances at width R (ms); the
// instances must be active with use_full set.  ids/begin scratch of at least
// ids.size() (+1) entries is passed in.
int time_width(const std::vector<SlotDesc>& h, SlotDesc* d_slots, const std::vector<int>& ids,
               bool f64, int R, int num_sms, int* d_ids, long long* d_begin,
               unsigned long long* d_counter, cudaStream_t s, float* ms) {
  std::vector<SlotDesc> tmp = h;
  std::vector<long long> begin(ids.size() + 1, 0);
  size_t smem = 0;
  for (size_t q = 0; q < ids.size(); ++q) {
    SlotDesc& sd = tmp[ids[q]];
    sd.R = R;
    sd.ntiles = tiles_at_width(sd.N, R);
    begin[q + 1] = begin[q] + (long long)sd.K * sd.ntiles;
    smem = std::max(smem, R == kResident ? resident_smem_bytes(f64, sd.d, sd.N)
                                         : gram_smem_bytes(f64, sd.d, R));
  }
  int per_sm = 0;
  const cudaError_t oe = R == kResident ? batch_resident_occupancy(f64, smem, &per_sm)
                                        : batch_score_occupancy(f64, R, smem, &per_sm);
  if (oe != cudaSuccess || per_sm < 1) return TRSTMI_ECUDA;
  const int grid = (int)std::min<long long>(begin.back(), (long long)num_sms * per_sm);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TRSTMI_ECUDA;
  int rc = TRSTMI_OK;
  if (cudaMemcpyAsync(d_slots, tmp.data(), sizeof(SlotDesc) * tmp.size(), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(d_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(d_begin, begin.data(), sizeof(long long) * begin.size(), cudaMemcpyHostToDevice, s))
    rc = TRSTMI_ECUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 5 && rc == TRSTMI_OK; ++rep) {
    float t = 0.f;
    if (cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s) ||
        cudaEventRecord(e0, s) ||
        (R == kResident
             ? launch_batch_resident(f64, d_slots, d_ids, d_begin, (int)ids.size(), begin.back(),
                                     d_counter, smem, grid, s, kPassFull)
             : launch_batch_score(f64, R, d_slots, d_ids, d_begin, (int)ids.size(), begin.back(),
                                  d_counter, smem, grid, s, kPassFull)) ||
        cudaEventRecord(e1, s) || cudaEventSynchronize(e1) || cudaEventElapsedTime(&t, e0, e1)) {
      rc = TRSTMI_ECUDA;
      break;
    }
    if (rep > 0) best = std::min(best, t);   // the first launch warms up
  }
  // restore the table
  if (cudaMemcpyAsync(d_slots, h.data(), sizeof(SlotDesc) * h.size(), cudaMemcpyHostToDevice, s))
    rc = TRSTMI_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  *ms = best;
  return rc;
}
}  // namespace trstmi

struct trstmi_batch {
  int n = 0;
  trstmi_options opt{};
  bool f64 = false, screen = false;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* block = nullptr;
  DeviceMemory dmem;   // where block, the plan and the scratch come from
  std::vector<int> N, d;
  std::vector<uint64_t> seed;
  std::vector<SlotDesc> h_slots;
  SlotDesc* d_slots = nullptr;
  uint32_t* d_err = nullptr;
  int* d_scratch_ids = nullptr;
  long long* d_scratch_begin = nullptr;
  BatchPlan plan;
  std::map<int, cudaGraphExec_t> graphs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

#define BTRY(expr)                                                          \
  do {                                                                      \
    if ((expr) != cudaSuccess) { cudaGetLastError(); return TRSTMI_ECUDA; } \
  } while (0)

// Chooses every instance's tile width: cached per (d, ceil log2 N), measured
// on the instances of a bucket when it is first seen.
int autotune(trstmi_batch* b) {
  const bool f64s = b->f64;   // width of the fp32 (or fp64) full pass
  std::map<std::pair<int, int>, std::vector<int>> buckets;
  for (int i = 0; i < b->n; ++i) buckets[{b->d[i], ceil_log2(b->N[i])}].push_back(i);
  // instances active with use_full while widths are timed (not advanced)
  k_batch_set_stop<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_slots, b->n, 1u);
  BTRY(cudaGetLastError());
  BTRY(launch_batch_begin(b->d_slots, b->n, b->plan.d_counters, BatchPlan::kCounters, f64s, false,
                          b->stream));
  // TRSTMI_TILE_WIDTH = 0 (whole candidates), 16, 32 or 64 fixes the choice
  // wherever it is feasible instead of timing the bucket (for measurements
  // that must reproduce a given configuration)
  int forced = -1;
  if (const char* env = std::getenv("TRSTMI_TILE_WIDTH")) {
    const int w = std::atoi(env);
    if (w == 0 || w == 16 || w == 32 || w == 64) forced = w / 16;
  }
  for (auto& kv : buckets) {
    int R = cached_width(f64s, kv.first.first, b->N[kv.second[0]]);
    if (forced >= 0) {
      bool ok = true;
      for (int i : kv.second) ok = ok && width_feasible(f64s, b->d[i], b->N[i], forced);
      R = ok ? forced : 1;
    } else if (R < 0) {
      float best = 1e30f;
      for (int cand : {kResident, 1, 2, 4}) {
        bool ok = true;
        for (int i : kv.second) ok = ok && width_feasible(f64s, b->d[i], b->N[i], cand);
        if (!ok) continue;
        float ms = 0.f;
        int rc = time_width(b->h_slots, b->d_slots, kv.second, f64s, cand, b->num_sms,
                            b->d_scratch_ids, b->d_scratch_begin, b->plan.d_counters, b->stream, &ms);
        if (rc) return rc;
        if (ms < best) { best = ms; R = cand; }
      }
      if (R < 0) R = 1;
      store_width(f64s, kv.first.first, b->N[kv.second[0]], R);
    }
    for (int i : kv.second) {
      b->h_slots[i].R = R;
      b->h_slots[i].ntiles = tiles_at_width(b->N[i], R);
    }
  }
  BTRY(cudaMemcpyAsync(b->d_slots, b->h_slots.data(), sizeof(SlotDesc) * b->n,
                       cudaMemcpyHostToDevice, b->stream));
  return b->plan.rebuild(b->h_slots, b->opt.precision, b->stream);
}

int batch_graph(trstmi_batch* b, int iters, cudaGraphExec_t* out) {
  auto it = b->graphs.find(iters);
  if (it != b->graphs.end()) { *out = it->second; return TRSTMI_OK; }
  cudaGraph_t g = nullptr;
  BTRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = TRSTMI_OK;
  for (int i = 0; i < iters && rc == TRSTMI_OK; ++i)
    rc = b->plan.enqueue_iteration(b->d_slots, b->n, b->d_err, b->stream);
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

// The instances' states are one contiguous array at the start of the arena.
int read_states(trstmi_batch* b, std::vector<DevState>* out) {
  out->resize(b->n);
  BTRY(cudaMemcpyAsync(out->data(), b->h_slots[0].st, sizeof(DevState) * b->n,
                       cudaMemcpyDeviceToHost, b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  return TRSTMI_OK;
}

}  // namespace

extern "C" {

void trstmi_batch_destroy(trstmi_batch_handle b) {
  if (!b) return;
  DeviceGuard device_guard(b->opt.device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->plan.destroy();
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  b->dmem.release(b->block);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int trstmi_batch_create(int n, const int* N, const int* d, const uint64_t* seeds,
                        const trstmi_options* opt, trstmi_batch_handle* out) {
  trstmi::TraceRange trace_range("trstmi_batch_create");
  if (!out) return TRSTMI_EINVAL;
  *out = nullptr;
  if (n < 1 || !N || !d || !seeds) return TRSTMI_EINVAL;
  trstmi_options o;
  if (opt) o = *opt; else trstmi_default_options(&o);
  if (o.precision < TRSTMI_FP64 || o.precision > TRSTMI_TF32_SCREEN) return TRSTMI_EINVAL;
  const bool screen = is_screen_prec(o.precision);
  if (o.K < 1 || o.trace_cap < 0 || !(o.delta0 > 0) || !(o.gamma_inc >= 1) ||
      !(o.gamma_dec > 0 && o.gamma_dec <= 1) || !(o.delta_min >= 0) ||
      !(o.delta_max >= o.delta_min) || !(o.screen_min_delta >= 0))
    return TRSTMI_EINVAL;
  if (screen && (o.topk < 1 || o.topk > 64 || o.topk > o.K)) return TRSTMI_EINVAL;
  if (!DeviceMemory::valid(o)) return TRSTMI_EINVAL;
  for (int i = 0; i < n; ++i)
    if (N[i] < 2 || d[i] < 1 || d[i] > kMaxD || (long long)N[i] * ((d[i] + 1) / 2) >= (1ll << 32))
      return TRSTMI_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return TRSTMI_ECUDA;
  if (o.device < 0 || o.device >= ndev) return TRSTMI_EINVAL;
  DeviceGuard device_guard(o.device);
  if (!device_guard.ok() || init_kernel_attributes() != cudaSuccess) return TRSTMI_ECUDA;

  trstmi_batch* b = new (std::nothrow) trstmi_batch();
  if (!b) return TRSTMI_ENOMEM;
  b->n = n; b->opt = o; b->f64 = (o.precision == TRSTMI_FP64); b->screen = screen;
  b->dmem = DeviceMemory(o);
  b->N.assign(N, N + n); b->d.assign(d, d + n); b->seed.assign(seeds, seeds + n);
  if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess) {
    delete b;
    return TRSTMI_ECUDA;
  }
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
    b->own_stream = true;
  } else {
    delete b;
    return TRSTMI_ECUDA;
  }
  // one arena: states, descriptors, error word, scratch tables, then per
  // instance frames, scores, trace and (screen modes) the certification scratch
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t K = (size_t)o.K, tcap = (size_t)std::max(o.trace_cap, 1);
  const size_t tk = screen ? (size_t)o.topk : 0;
  size_t off = 0;
  const size_t o_st = off; off = up(off + sizeof(DevState) * n);
  const size_t o_sl = off; off = up(off + sizeof(SlotDesc) * n);
  const size_t o_er = off; off = up(off + sizeof(uint32_t));
  const size_t o_ids = off; off = up(off + sizeof(int) * n);
  const size_t o_beg = off; off = up(off + sizeof(long long) * (n + 1));
  std::vector<size_t> o_phi64(n), o_phi32(n), o_mu2(n), o_tr(n), o_scr(n);
  for (int i = 0; i < n; ++i) {
    const size_t nd = (size_t)N[i] * d[i];
    o_phi64[i] = off; off = up(off + nd * sizeof(double2));
    o_phi32[i] = off; off = up(off + nd * sizeof(float2));
    o_mu2[i] = off; off = up(off + K * sizeof(unsigned long long));
    o_tr[i] = off; off = up(off + tcap * sizeof(TraceRowDev));
    if (screen) {
      o_scr[i] = off;
      off += 2 * up(tk * sizeof(uint32_t)) + up(nd * sizeof(double2)) +
            up(nd * sizeof(float2)) + up(4 * sizeof(uint32_t)) + up(sizeof(unsigned long long)) +
            up((size_t)slot_pair_cap(N[i]) * sizeof(uint2));
    }
  }
  // scratch for drawing the candidates of the large binary32 instances once
  // per pass (the largest such instance's candidates, at most 512 MiB)
  size_t planes_bytes = 0;
  if (o.precision != TRSTMI_FP64)
    for (int i = 0; i < n; ++i) {
      const size_t need = std::max<size_t>((size_t)o.K, tk) * 2 * (size_t)d[i] *
                          (size_t)N[i] * sizeof(float);
      if (N[i] >= BatchPlan::kPlanesMinN && need <= kBatchPlanesMax)
        planes_bytes = std::max(planes_bytes, need);
    }
  b->plan.dmem = b->dmem;
  if (b->dmem.allocate(&b->block, off) != cudaSuccess ||
      b->plan.init(n, screen ? (long long)n * o.K : 0, b->num_sms, planes_bytes) != TRSTMI_OK) {
    cudaGetLastError();
    trstmi_batch_destroy(b);
    return TRSTMI_ENOMEM;
  }
  char* base = (char*)b->block;
  DevState* states = (DevState*)(base + o_st);
  b->d_slots = (SlotDesc*)(base + o_sl);
  b->d_err = (uint32_t*)(base + o_er);
  b->d_scratch_ids = (int*)(base + o_ids);
  b->d_scratch_begin = (long long*)(base + o_beg);
  b->h_slots.resize(n);
  std::vector<DevState> s0(n);
  for (int i = 0; i < n; ++i) {
    const size_t nd = (size_t)N[i] * d[i];
    SlotDesc& sd = b->h_slots[i];
    std::memset(&sd, 0, sizeof(sd));
    sd.st = states + i;
    double2* p64 = (double2*)(base + o_phi64[i]);
    float2* p32 = (float2*)(base + o_phi32[i]);
    sd.phi = b->f64 ? (void*)p64 : (void*)p32;
    sd.phi_other = b->f64 ? (void*)p32 : (void*)p64;
    sd.mu2 = base + o_mu2[i];
    sd.trace = (TraceRowDev*)(base + o_tr[i]);
    sd.seed = seeds[i];
    sd.N = N[i]; sd.d = d[i]; sd.K = o.K; sd.R = 1; sd.ntiles = ntiles_for(N[i], 1);
    if (screen) {
      char* q = base + o_scr[i];
      sd.screen = screen_supported(N[i], d[i], screen_fmt_of(o.precision, d[i])) ? 1 : 0;
      sd.topk = (uint32_t*)q; q += up(tk * sizeof(uint32_t));
      sd.mu2_top = (unsigned int*)q; q += up(tk * sizeof(uint32_t));
      sd.cand64 = (double2*)q; q += up(nd * sizeof(double2));
      sd.cand32 = (float2*)q; q += up(nd * sizeof(float2));
      sd.cert32 = (unsigned int*)q; q += up(4 * sizeof(uint32_t));
      sd.cert64 = (unsigned long long*)q; q += up(sizeof(unsigned long long));
      sd.pairs = (uint2*)q;
      sd.topk_n = o.topk;
      sd.pair_cap = slot_pair_cap(sd.N);
    }
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
    cudaError_t e;
    if (screen) {          // certified in binary64 as the standalone instance does
      e = launch_frame_certify(N[i], d[i], p64, p32, sd.cert32, sd.cert64, sd.pairs, sd.pair_cap,
                               &sd.st->npairs, &sd.st->overflow, nullptr, b->num_sms, s);
    } else {
      src.phi = sd.phi;
      e = b->f64 ? launch_gram_f64(N[i], d[i], 1, src, (unsigned long long*)sd.mu2, b->num_sms, s)
                 : launch_gram_f32(N[i], d[i], 1, src, (unsigned int*)sd.mu2, nullptr, b->num_sms, s);
    }
    if (e != cudaSuccess) rc = TRSTMI_ECUDA;
  }
  if (rc == TRSTMI_OK) {
    if (screen) k_batch_set_mu2cur_cert<<<(n + 127) / 128, 128, 0, s>>>(b->d_slots, n);
    else if (b->f64) k_batch_set_mu2cur<unsigned long long><<<(n + 127) / 128, 128, 0, s>>>(b->d_slots, n);
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
  trstmi::TraceRange trace_range("trstmi_batch_step");
  if (!b || iters < 0) return TRSTMI_EINVAL;
  DeviceGuard device_guard(b->opt.device);
  if (!device_guard.ok()) return TRSTMI_ECUDA;
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
  BTRY(cudaMemcpy(&err, b->d_err, sizeof(err), cudaMemcpyDeviceToHost));
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
  DeviceGuard device_guard(b->opt.device);
  if (!device_guard.ok()) return TRSTMI_ECUDA;
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
  DeviceGuard device_guard(b->opt.device);
  if (!device_guard.ok()) return TRSTMI_ECUDA;
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
  DeviceGuard device_guard(b->opt.device);
  if (!device_guard.ok()) return TRSTMI_ECUDA;
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
  DeviceGuard device_guard(b->opt.device);
  if (!device_guard.ok()) return TRSTMI_ECUDA;
  cudaStream_t s = b->stream;
  void* flush = nullptr;
  if (flush_bytes) BTRY(b->dmem.allocate(&flush, flush_bytes));
  double total = 0.0;
  int rc = TRSTMI_OK;
  for (int l = 0; l < launches && rc == TRSTMI_OK; ++l) {
    // every instance active for one iteration, not advanced; the screen modes
    // time the screen (all instances screened), the others the full pass
    k_batch_set_stop<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_slots, b->n, 1u);
    if (cudaGetLastError() != cudaSuccess ||
        launch_batch_begin(b->d_slots, b->n, b->plan.d_counters, BatchPlan::kCounters, b->f64,
                           b->screen, s) ||
        (flush && cudaMemsetAsync(flush, l & 0xff, flush_bytes, s)) ||
        cudaEventRecord(b->ev0, s) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    cudaError_t e = b->screen
        ? b->plan.launch_screen(b->d_err, s)
        : b->plan.launch_pass(kPassFull, b->d_slots, s);
    if (e == cudaSuccess && !b->screen) e = b->plan.launch_large(kPassFull, s);
    float ms = 0.f;
    if (e != cudaSuccess || cudaEventRecord(b->ev1, s) != cudaSuccess ||
        cudaEventSynchronize(b->ev1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, b->ev0, b->ev1) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    total += ms;
  }
  b->dmem.release(flush);
  if (rc == TRSTMI_OK) *avg_ms = total / launches;
  return rc;
}

int trstmi_batch_tile_widths(trstmi_batch_handle b, int* widths) {
  if (!b || !widths) return TRSTMI_EINVAL;
  for (int i = 0; i < b->n; ++i) widths[i] = 16 * b->h_slots[i].R;   // 0: whole candidate
  return TRSTMI_OK;
}

}  // extern "C"
