// Serving loop (trstmi_server_*, trstmi_submit / trstmi_poll, include/trstmi.h).
//
// A host scheduler thread keeps a set of resident search slots on one GPU and
// advances all of them together: each round is `iters_per_round` iterations
// of the shared batched launches of BatchPlan (iteration start, the
// tensor-core screen in the screen modes, persistent scoring passes over
// every slot's (candidate, tile) work items, per-slot certification, accept
// rule and commit).  Requests wait in a FIFO queue; the head is admitted as soon as a
// slot and enough of the device-memory budget are free (continuous
// batching).  A slot retires at a round boundary once its search reached its
// target, spent its iteration budget or was cancelled.  Each slot keeps its
// own state, seed and counters, so a request's result is exactly the one the
// same search gives alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/trstmi.h"
#include "trace.h"
#include "kernels.h"

using namespace trstmi;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over one device allocation (the HBM budget).
class Arena {
 public:
  void reset(char* base, size_t size) {
    base_ = base;
    size_ = size;
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return base_; }
  size_t used() const { return used_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Req {
  trstmi_request req{};
  double target = -1.0;
  int status = TRSTMI_PENDING;
  bool cancel = false;
  int64_t t_submit = 0, t_admit = 0, t_done = 0;
  double mu = 0.0, welch = 0.0;
  int32_t iters = 0, accepts = 0, reached = 0;
  uint64_t pairs = 0;
  std::vector<double> phi;
};

struct Slot {
  uint64_t ticket = 0;
  size_t off = 0, bytes = 0;
  int state_idx = -1;
  SlotDesc desc{};
  uint32_t budget = 0;
  uint64_t pairs = 0;   // pairs scored per iteration, K N(N-1)/2
};

uint64_t pairs_per_iteration(int K, int N) {
  return (uint64_t)K * ((uint64_t)N * (uint64_t)(N - 1) / 2);
}

double welch_bound(int N, int d) {
  if (N <= d || N < 2) return 0.0;
  return std::sqrt((double)(N - d) / ((double)d * (double)(N - 1)));
}

__global__ void k_srv_set_stop(SlotDesc* slots, int n, uint32_t iters, const uint32_t* budget) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  DevState* st = slots[s].st;
  unsigned long long stop = (unsigned long long)st->t + iters;
  if (stop > budget[s]) stop = budget[s];
  st->t_stop = (uint32_t)stop;
  st->t_call = st->t;   // iterations of this round = t - t_call
  st->accepts_call = st->accepts;
}

// Marks a slot active (or not) for a width measurement, without advancing it.
__global__ void k_srv_activate(DevState* st, uint32_t on) {
  st->active = on;
  st->use_full = on;
  st->delta_used = st->delta;
}

template <typename B>
__global__ void k_srv_set_mu2cur(DevState* st, const void* mu2) {
  st->mu2_cur = (double)nonneg_from_bits(reinterpret_cast<const B*>(mu2)[0]);
  st->done = (st->mu2_cur <= st->target2) ? 1u : 0u;
}

// Pair list of the certification: the standalone instance's 65536 pairs, or
// every pair when there are fewer, so that the list overflows exactly when a
// standalone run's does.
uint32_t slot_pair_cap(int N) {
  const unsigned long long all = (unsigned long long)N * (unsigned long long)(N - 1) / 2;
  return (uint32_t)std::min<unsigned long long>(all, 1ull << 16);
}

bool is_screen_prec(int p) { return is_screen_precision(p); }

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Screen modes: top-k indices and scores, the binary64 winner and its binary32
// rounding, the certification words and the preselected pair list.
size_t screen_bytes(int N, int d, int topk) {
  const size_t nd = (size_t)N * d;
  return 2 * up256((size_t)topk * sizeof(uint32_t)) + up256(nd * sizeof(double2)) +
         up256(nd * sizeof(float2)) + up256(4 * sizeof(uint32_t)) +
         up256(sizeof(unsigned long long)) + up256((size_t)slot_pair_cap(N) * sizeof(uint2));
}

size_t slot_bytes(int N, int d, const trstmi_options& o) {
  const size_t nd = (size_t)N * d;
  size_t b = up256(nd * sizeof(double2)) + up256(nd * sizeof(float2)) + up256((size_t)o.K * 8) +
             up256((size_t)std::max(o.trace_cap, 1) * sizeof(TraceRowDev));
  if (is_screen_prec(o.precision)) b += screen_bytes(N, d, o.topk);
  return b;
}

}  // namespace

struct trstmi_server {
  trstmi_server_opts opt{};
  bool f64 = false, screen = false;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* arena_mem = nullptr;
  DeviceMemory dmem;                  // where the tables, arena and plan come from
  Arena arena;
  DevState* d_states = nullptr;       // max_slots states
  SlotDesc* d_slots = nullptr;        // active slot table
  uint32_t* d_budget = nullptr;
  uint32_t* d_err = nullptr;          // screen kernel's abort word
  int* d_tune_ids = nullptr;          // width measurement: one-slot group table
  long long* d_tune_begin = nullptr;
  std::vector<int> free_states;
  std::vector<Slot> slots;
  uint64_t resident_pairs = 0;
  BatchPlan plan;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::atomic<int> active_count{0};
  int worker_error = TRSTMI_OK;
  std::thread worker;
  // statistics
  uint64_t submitted = 0, admitted = 0, completed = 0, cancelled = 0, rounds = 0;
  int32_t timed_out = 0;
  uint64_t pairs_scored = 0;
  double gpu_busy_s = 0.0;
  std::atomic<uint64_t> launches{0};   // kernels the loop launched
};

namespace {

int choose_width(trstmi_server* sv, Slot& sl) {
  const int N = sl.desc.N, d = sl.desc.d;
  int R = cached_width(sv->f64, d, N);   // the binary32 pass in the screen modes
  if (R >= 0) return R;
  // large binary32 searches draw their candidates once into the plan's
  // scratch and take the widest tiles; nothing to measure
  if (!sv->f64 && N >= BatchPlan::kPlanesMinN && width_feasible(false, d, N, 4)) {
    store_width(false, d, N, 4);
    return 4;
  }
  // measure this bucket on this slot alone (its state is active for timing)
  int best_R = 1;
  float best = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 1;
  k_srv_activate<<<1, 1, 0, sv->stream>>>(sl.desc.st, 1u);
  sv->launches += 2;   // this one and the deactivation below
  for (int cand : {kResident, 1, 2, 4}) {
    if (!width_feasible(sv->f64, d, N, cand)) continue;
    SlotDesc tmp = sl.desc;
    tmp.R = cand;
    tmp.ntiles = tiles_at_width(N, cand);
    const long long nitems = (long long)tmp.K * tmp.ntiles;
    const long long begin[2] = {0, nitems};
    const int ids[1] = {0};
    const size_t smem = cand == kResident ? resident_smem_bytes(sv->f64, d, N)
                                          : gram_smem_bytes(sv->f64, d, cand);
    int per_sm = 0;
    const cudaError_t oe = cand == kResident ? batch_resident_occupancy(sv->f64, smem, &per_sm)
                                             : batch_score_occupancy(sv->f64, cand, smem, &per_sm);
    if (oe != cudaSuccess || per_sm < 1) continue;
    const int grid = (int)std::min<long long>(nitems, (long long)sv->num_sms * per_sm);
    // slot table entry 0 is rewritten by rebuild_tables before the next round
    cudaMemcpyAsync(sv->d_slots, &tmp, sizeof(SlotDesc), cudaMemcpyHostToDevice, sv->stream);
    cudaMemcpyAsync(sv->d_tune_ids, ids, sizeof(ids), cudaMemcpyHostToDevice, sv->stream);
    cudaMemcpyAsync(sv->d_tune_begin, begin, sizeof(begin), cudaMemcpyHostToDevice, sv->stream);
    float t_best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaMemsetAsync(sv->plan.d_counters, 0, sizeof(unsigned long long), sv->stream);
      cudaEventRecord(e0, sv->stream);
      if (cand == kResident)
        launch_batch_resident(sv->f64, sv->d_slots, sv->d_tune_ids, sv->d_tune_begin, 1, nitems,
                              sv->plan.d_counters, smem, grid, sv->stream, kPassFull);
      else
        launch_batch_score(sv->f64, cand, sv->d_slots, sv->d_tune_ids, sv->d_tune_begin, 1, nitems,
                           sv->plan.d_counters, smem, grid, sv->stream, kPassFull);
      cudaEventRecord(e1, sv->stream);
      sv->launches += 1;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) t_best = std::min(t_best, ms);
    }
    if (t_best < best) { best = t_best; best_R = cand; }
  }
  k_srv_activate<<<1, 1, 0, sv->stream>>>(sl.desc.st, 0u);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  store_width(sv->f64, d, N, best_R);
  return best_R;
}

// Device tables for the current active set: descriptors, budgets, launch plan.
int rebuild_tables(trstmi_server* sv) {
  const int n = (int)sv->slots.size();
  std::vector<SlotDesc> h(n);
  std::vector<uint32_t> budget(n);
  for (int i = 0; i < n; ++i) {
    h[i] = sv->slots[i].desc;
    budget[i] = sv->slots[i].budget;
  }
  int rc = sv->plan.rebuild(h, sv->opt.search.precision, sv->stream);
  if (rc) return rc;
  if (n > 0 &&
      (cudaMemcpyAsync(sv->d_slots, h.data(), sizeof(SlotDesc) * n, cudaMemcpyHostToDevice,
                       sv->stream) != cudaSuccess ||
       cudaMemcpyAsync(sv->d_budget, budget.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice,
                       sv->stream) != cudaSuccess))
    return TRSTMI_ECUDA;
  return TRSTMI_OK;
}

// Sets up the slot of a request: memory, state, seeded frame, initial score.
int admit(trstmi_server* sv, uint64_t ticket, Req& r, Slot* out) {
  const trstmi_options& o = sv->opt.search;
  const int N = r.req.N, d = r.req.d;
  Slot sl;
  sl.ticket = ticket;
  sl.bytes = slot_bytes(N, d, o);
  if (!sv->arena.alloc(sl.bytes, &sl.off)) return TRSTMI_ENOMEM;
  sl.state_idx = sv->free_states.back();
  sv->free_states.pop_back();
  char* p = sv->arena.base() + sl.off;
  const size_t nd = (size_t)N * d;
  double2* p64 = (double2*)p;
  float2* p32 = (float2*)(p + up256(nd * sizeof(double2)));
  void* mu2 = p + up256(nd * sizeof(double2)) + up256(nd * sizeof(float2));
  TraceRowDev* tr = (TraceRowDev*)((char*)mu2 + up256((size_t)o.K * 8));
  SlotDesc& sd = sl.desc;
  std::memset(&sd, 0, sizeof(sd));
  if (sv->screen) {
    char* q = (char*)tr + up256((size_t)std::max(o.trace_cap, 1) * sizeof(TraceRowDev));
    sd.screen = screen_supported(N, d, screen_fmt_of(o.precision, d)) ? 1 : 0;
    sd.topk = (uint32_t*)q; q += up256((size_t)o.topk * sizeof(uint32_t));
    sd.mu2_top = (unsigned int*)q; q += up256((size_t)o.topk * sizeof(uint32_t));
    sd.cand64 = (double2*)q; q += up256(nd * sizeof(double2));
    sd.cand32 = (float2*)q; q += up256(nd * sizeof(float2));
    sd.cert32 = (unsigned int*)q; q += up256(4 * sizeof(uint32_t));
    sd.cert64 = (unsigned long long*)q; q += up256(sizeof(unsigned long long));
    sd.pairs = (uint2*)q;
    sd.topk_n = o.topk;
    sd.pair_cap = slot_pair_cap(N);
  }
  sd.st = sv->d_states + sl.state_idx;
  sd.phi = sv->f64 ? (void*)p64 : (void*)p32;
  sd.phi_other = sv->f64 ? (void*)p32 : (void*)p64;
  sd.mu2 = mu2;
  sd.trace = tr;
  sd.seed = r.req.seed;
  sd.N = N; sd.d = d; sd.K = o.K;
  sl.budget = (uint32_t)std::max(0, r.req.budget_iters);
  sl.pairs = pairs_per_iteration(o.K, N);
  DevState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.delta = o.delta0; s0.delta_used = o.delta0;
  s0.target2 = r.target > 0 ? r.target * r.target : -1.0;
  s0.gamma_inc = o.gamma_inc; s0.gamma_dec = o.gamma_dec;
  s0.delta_min = o.delta_min; s0.delta_max = o.delta_max;
  s0.screen_min_delta = o.screen_min_delta;
  s0.trace_cap = (uint32_t)o.trace_cap;
  cudaStream_t s = sv->stream;
  if (cudaMemsetAsync(p, 0, sl.bytes, s) != cudaSuccess ||
      cudaMemcpyAsync(sd.st, &s0, sizeof(s0), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      launch_init_frame(N, d, sd.seed, p64, p32, sd.st, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  // initial score in the deciding precision (binary64 in the screen modes,
  // certified by the same passes as the standalone instance's)
  GramSource src{};
  src.perturb = false;
  src.phi = sd.phi;
  void* init_out = sv->screen ? (void*)sd.cert64 : mu2;
  cudaError_t e =
      sv->screen ? launch_frame_certify(N, d, p64, p32, sd.cert32, sd.cert64, sd.pairs,
                                        sd.pair_cap, &sd.st->npairs, &sd.st->overflow, nullptr,
                                        sv->num_sms, s)
      : sv->f64  ? launch_gram_f64(N, d, 1, src, (unsigned long long*)init_out, sv->num_sms, s)
                 : launch_gram_f32(N, d, 1, src, (unsigned int*)init_out, nullptr, sv->num_sms, s);
  if (e != cudaSuccess) return TRSTMI_ECUDA;
  if (sv->f64 || sv->screen) k_srv_set_mu2cur<unsigned long long><<<1, 1, 0, s>>>(sd.st, init_out);
  else k_srv_set_mu2cur<unsigned int><<<1, 1, 0, s>>>(sd.st, init_out);
  if (cudaGetLastError() != cudaSuccess) return TRSTMI_ECUDA;
  // initial frame, initial score (four certification passes in the screen
  // modes), its copy into the state
  sv->launches += sv->screen ? 6 : 3;
  // tile width: the cached choice for this (d, N) bucket, measured if new
  sd.R = 1;
  sd.ntiles = tiles_at_width(N, 1);
  const int R = choose_width(sv, sl);
  sd.R = R;
  sd.ntiles = tiles_at_width(N, R);
  *out = sl;
  return TRSTMI_OK;
}

// a request past its deadline (deadline_ms after submission)
bool expired(const Req& r, int64_t now) {
  return r.req.deadline_ms > 0.0 && (double)(now - r.t_submit) > r.req.deadline_ms * 1e6;
}

void retire(trstmi_server* sv, size_t k, const DevState& st, int status) {
  Slot& sl = sv->slots[k];
  Req& r = sv->reqs[sl.ticket];
  r.mu = std::sqrt(st.mu2_cur);
  r.welch = welch_bound(r.req.N, r.req.d);
  r.iters = (int32_t)st.t;
  r.accepts = (int32_t)st.accepts;
  r.reached = (int32_t)st.done;
  r.pairs = (uint64_t)st.t * (uint64_t)sl.desc.K * ((uint64_t)r.req.N * (r.req.N - 1) / 2);
  if (r.req.want_phi && status == TRSTMI_OK) {
    r.phi.resize((size_t)2 * r.req.N * r.req.d);
    const void* p64 = sv->f64 ? sl.desc.phi : sl.desc.phi_other;
    if (cudaMemcpyAsync(r.phi.data(), p64, r.phi.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        sv->stream) != cudaSuccess ||
        cudaStreamSynchronize(sv->stream) != cudaSuccess)
      status = TRSTMI_ECUDA;
  }
  r.status = status;
  r.t_done = now_ns();
  sv->arena.release(sl.off, sl.bytes);
  sv->resident_pairs -= sl.pairs;
  sv->free_states.push_back(sl.state_idx);
  sv->slots.erase(sv->slots.begin() + k);
  sv->active_count = (int)sv->slots.size();
  if (status == TRSTMI_ECANCELLED) ++sv->cancelled;
  else if (status == TRSTMI_ETIMEOUT) ++sv->timed_out;
  else ++sv->completed;
}

void worker_main(trstmi_server* sv) {
  cudaSetDevice(sv->opt.search.device);
  std::deque<uint64_t> pending;
  bool changed = true;
  std::vector<DevState> st, all_st;
  const int I = std::max(1, sv->opt.iters_per_round);
  while (!sv->stop.load()) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (sv->slots.empty() && pending.empty() && sv->queue.empty())
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      while (!sv->queue.empty()) { pending.push_back(sv->queue.front()); sv->queue.pop_front(); }
      // drop cancelled and expired requests that never started
      const int64_t now = now_ns();
      for (auto it = pending.begin(); it != pending.end();) {
        Req& r = sv->reqs[*it];
        if (r.cancel || expired(r, now)) {
          r.status = r.cancel ? TRSTMI_ECANCELLED : TRSTMI_ETIMEOUT;
          r.t_done = now;
          if (r.cancel) ++sv->cancelled; else ++sv->timed_out;
          it = pending.erase(it);
          sv->cv_done.notify_all();
        } else {
          ++it;
        }
      }
    }
    if (sv->stop.load()) break;
    // admission, FIFO: the head waits until a slot and its memory are free
    while (!pending.empty() && (int)sv->slots.size() < sv->opt.max_slots) {
      const uint64_t tk = pending.front();
      Req* r;
      {
        std::lock_guard<std::mutex> g(sv->mu);
        r = &sv->reqs[tk];
      }
      // resident work cap: the head waits for running searches to retire
      const uint64_t cap = sv->opt.max_resident_pairs;
      if (cap && !sv->slots.empty() &&
          sv->resident_pairs + pairs_per_iteration(sv->opt.search.K, r->req.N) > cap)
        break;
      Slot sl;
      const int rc = admit(sv, tk, *r, &sl);
      if (rc == TRSTMI_ENOMEM) {
        if (sv->slots.empty()) {   // can never fit the budget
          std::lock_guard<std::mutex> g(sv->mu);
          r->status = TRSTMI_ENOMEM;
          r->t_done = now_ns();
          pending.pop_front();
          sv->cv_done.notify_all();
          continue;
        }
        break;
      }
      if (rc) { sv->worker_error = rc; sv->stop = true; break; }
      {
        std::lock_guard<std::mutex> g(sv->mu);
        r->t_admit = now_ns();
        ++sv->admitted;
      }
      pending.pop_front();
      sv->resident_pairs += sl.pairs;
      sv->slots.push_back(sl);
      sv->active_count = (int)sv->slots.size();
      changed = true;
    }
    if (sv->stop.load()) break;
    if (sv->slots.empty()) continue;
    if (changed) {
      if (rebuild_tables(sv) != TRSTMI_OK) { sv->worker_error = TRSTMI_ECUDA; break; }
      changed = false;
    }
    // one round: I iterations of every active slot, shared launches
    trstmi::TraceRange trace_range("server round");
    const int n = (int)sv->slots.size();
    const int64_t t0 = now_ns();
    cudaStream_t s = sv->stream;
    k_srv_set_stop<<<(n + 127) / 128, 128, 0, s>>>(sv->d_slots, n, (uint32_t)I, sv->d_budget);
    bool ok = cudaGetLastError() == cudaSuccess;
    for (int it = 0; ok && it < I; ++it)
      ok = sv->plan.enqueue_iteration(sv->d_slots, n, sv->d_err, s) == TRSTMI_OK;
    sv->launches += 1 + (uint64_t)I * (uint64_t)sv->plan.kernels_per_iteration();
    // one copy of the whole state array, then each slot's entry
    all_st.resize(sv->opt.max_slots);
    ok = ok && cudaMemcpyAsync(all_st.data(), sv->d_states, sizeof(DevState) * all_st.size(),
                               cudaMemcpyDeviceToHost, s) == cudaSuccess;
    uint32_t screen_err = 0;
    ok = ok && cudaMemcpyAsync(&screen_err, sv->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                               s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    st.resize(n);
    for (int k = 0; ok && k < n; ++k) st[k] = all_st[sv->slots[k].state_idx];
    // a screen launch that gave up waiting aborts every slot of the round
    if (ok && screen_err) {
      for (int k = 0; k < n; ++k) st[k].error |= screen_err;
      ok = cudaMemsetAsync(sv->d_err, 0, sizeof(uint32_t), s) == cudaSuccess;
    }
    if (!ok) { cudaGetLastError(); sv->worker_error = TRSTMI_ECUDA; break; }
    {
      std::lock_guard<std::mutex> g(sv->mu);
      sv->gpu_busy_s += (now_ns() - t0) * 1e-9;
      ++sv->rounds;
      for (int k = 0; k < n; ++k)
        sv->pairs_scored += (uint64_t)(st[k].t - st[k].t_call) * (uint64_t)sv->slots[k].desc.K *
                            ((uint64_t)sv->slots[k].desc.N * (sv->slots[k].desc.N - 1) / 2);
      const int64_t now = now_ns();
      for (int k = n - 1; k >= 0; --k) {
        const Req& r = sv->reqs[sv->slots[k].ticket];
        const uint32_t err = st[k].error;
        if (err) {
          retire(sv, k, st[k], (err & kErrTimeout) ? TRSTMI_ETIMEOUT : TRSTMI_EINVAL);
          changed = true;
        } else if (r.cancel) {
          retire(sv, k, st[k], TRSTMI_ECANCELLED);
          changed = true;
        } else if (st[k].done || st[k].t >= sv->slots[k].budget) {
          retire(sv, k, st[k], TRSTMI_OK);
          changed = true;
        } else if (expired(r, now)) {
          retire(sv, k, st[k], TRSTMI_ETIMEOUT);
          changed = true;
        }
      }
      sv->cv_done.notify_all();
    }
  }
  // fail whatever is left
  std::lock_guard<std::mutex> g(sv->mu);
  for (auto& kv : sv->reqs)
    if (kv.second.status == TRSTMI_PENDING) {
      kv.second.status = sv->worker_error ? sv->worker_error : TRSTMI_ECANCELLED;
      kv.second.t_done = now_ns();
    }
  sv->cv_done.notify_all();
}

void fill_result(const Req& r, trstmi_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = r.status;
  out->iters = r.iters;
  out->accepts = r.accepts;
  out->reached_target = r.reached;
  out->mu = r.mu;
  out->welch = r.welch;
  out->t_submit_ns = r.t_submit;
  out->t_admit_ns = r.t_admit;
  out->t_done_ns = r.t_done;
  out->pairs_scored = r.pairs;
}

}  // namespace

extern "C" {

void trstmi_default_server_opts(trstmi_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  trstmi_default_options(&o->search);
  o->search.precision = TRSTMI_FP32;
  o->search.K = 8;
  o->search.trace_cap = 0;
  o->hbm_budget = (size_t)4 << 30;
  o->max_slots = 256;
  o->iters_per_round = 20;
  o->queue_cap = 1 << 16;
  o->max_resident_pairs = 1ull << 28;
}

void trstmi_server_destroy(trstmi_server* sv) {
  if (!sv) return;
  sv->stop = true;
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  DeviceGuard device_guard(sv->opt.search.device);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  sv->plan.destroy();
  sv->dmem.release(sv->arena_mem);
  sv->dmem.release(sv->d_states);
  if (sv->own_stream && sv->stream) cudaStreamDestroy(sv->stream);
  delete sv;
}

int trstmi_server_create(const trstmi_server_opts* opts, trstmi_server** out) {
  if (!out) return TRSTMI_EINVAL;
  *out = nullptr;
  trstmi_server_opts o;
  if (opts) o = *opts; else trstmi_default_server_opts(&o);
  const trstmi_options& so = o.search;
  if (so.precision < TRSTMI_FP64 || so.precision > TRSTMI_TF32_SCREEN) return TRSTMI_EINVAL;
  if (o.max_slots < 1 || o.max_slots > 65536 || o.queue_cap < 1 || o.iters_per_round < 1 ||
      so.K < 1 || so.trace_cap < 0 || o.hbm_budget < 4096 || !(so.delta0 > 0) ||
      !(so.gamma_inc >= 1) || !(so.gamma_dec > 0 && so.gamma_dec <= 1) || !(so.delta_min >= 0) ||
      !(so.delta_max >= so.delta_min) || !(so.screen_min_delta >= 0))
    return TRSTMI_EINVAL;
  if (is_screen_prec(so.precision) && (so.topk < 1 || so.topk > 64 || so.topk > so.K))
    return TRSTMI_EINVAL;
  if (!DeviceMemory::valid(so)) return TRSTMI_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return TRSTMI_ECUDA;
  if (so.device < 0 || so.device >= ndev) return TRSTMI_EINVAL;
  DeviceGuard device_guard(so.device);
  if (!device_guard.ok() || init_kernel_attributes() != cudaSuccess) return TRSTMI_ECUDA;
  trstmi_server* sv = new (std::nothrow) trstmi_server();
  if (!sv) return TRSTMI_ENOMEM;
  sv->opt = o;
  sv->dmem = DeviceMemory(so);
  sv->f64 = so.precision == TRSTMI_FP64;
  sv->screen = is_screen_prec(so.precision);
  if (cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, so.device) != cudaSuccess) {
    delete sv;
    return TRSTMI_ECUDA;
  }
  if (so.stream) {
    sv->stream = (cudaStream_t)so.stream;
  } else if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) == cudaSuccess) {
    sv->own_stream = true;
  } else {
    delete sv;
    return TRSTMI_ECUDA;
  }
  // control tables (states, descriptors, budgets, error word, width measurement)
  const size_t ms = (size_t)o.max_slots;
  const size_t b_st = up256(ms * sizeof(DevState)), b_sl = up256(ms * sizeof(SlotDesc)),
               b_bu = up256(ms * sizeof(uint32_t)), b_er = up256(sizeof(uint32_t)),
               b_ti = up256(sizeof(int)), b_tb = up256(2 * sizeof(long long));
  // of the budget, min(1/8, 256 MiB) is the scratch in which the candidates
  // of large binary32 searches are drawn once per pass; the rest holds the
  // resident searches
  const size_t planes_bytes =
      sv->f64 ? 0 : std::min<size_t>(256ull << 20, o.hbm_budget / 8) / 256 * 256;
  const size_t arena_bytes = o.hbm_budget - planes_bytes;
  char* ctl = nullptr;
  sv->plan.dmem = sv->dmem;
  if (sv->dmem.allocate(reinterpret_cast<void**>(&ctl), b_st + b_sl + b_bu + b_er + b_ti + b_tb) !=
          cudaSuccess ||
      cudaMemset(ctl, 0, b_st + b_sl + b_bu + b_er + b_ti + b_tb) != cudaSuccess ||
      sv->dmem.allocate(&sv->arena_mem, arena_bytes) != cudaSuccess ||
      sv->plan.init(o.max_slots, sv->screen ? (long long)o.max_slots * so.K : 0, sv->num_sms,
                    planes_bytes) != TRSTMI_OK) {
    cudaGetLastError();
    sv->d_states = (DevState*)ctl;   // freed by destroy
    trstmi_server_destroy(sv);
    return TRSTMI_ENOMEM;
  }
  sv->d_states = (DevState*)ctl;
  sv->d_slots = (SlotDesc*)(ctl + b_st);
  sv->d_budget = (uint32_t*)(ctl + b_st + b_sl);
  sv->d_err = (uint32_t*)(ctl + b_st + b_sl + b_bu);
  sv->d_tune_ids = (int*)(ctl + b_st + b_sl + b_bu + b_er);
  sv->d_tune_begin = (long long*)(ctl + b_st + b_sl + b_bu + b_er + b_ti);
  sv->arena.reset((char*)sv->arena_mem, arena_bytes);
  for (int i = o.max_slots - 1; i >= 0; --i) sv->free_states.push_back(i);
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return TRSTMI_OK;
}

int trstmi_submit(trstmi_server* sv, const trstmi_request* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return TRSTMI_EINVAL;
  if (req->N < 2 || req->d < 1 || req->d > kMaxD || req->budget_iters < 0 ||
      (long long)req->N * ((req->d + 1) / 2) >= (1ll << 32) || !(req->deadline_ms >= 0.0) ||
      !(req->deadline_ms < INFINITY))
    return TRSTMI_EINVAL;
  std::lock_guard<std::mutex> g(sv->mu);
  if (sv->worker_error) return sv->worker_error;
  if ((int)sv->queue.size() >= sv->opt.queue_cap) return TRSTMI_EBUSY;
  const uint64_t tk = sv->next_ticket++;
  Req& r = sv->reqs[tk];
  r.req = *req;
  r.target = req->target_mu > 0 ? req->target_mu
           : (req->target_rel_welch > 0 ? req->target_rel_welch * welch_bound(req->N, req->d) : -1.0);
  r.t_submit = now_ns();
  sv->queue.push_back(tk);
  ++sv->submitted;
  *ticket = tk;
  sv->cv_work.notify_one();
  return TRSTMI_OK;
}

int trstmi_poll(trstmi_server* sv, uint64_t ticket, trstmi_result* out, double* phi_out) {
  if (!sv || !out) return TRSTMI_EINVAL;
  std::lock_guard<std::mutex> g(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return TRSTMI_ENOTFOUND;
  const Req& r = it->second;
  fill_result(r, out);
  if (r.status == TRSTMI_PENDING) return TRSTMI_PENDING;
  if (phi_out && !r.phi.empty()) std::memcpy(phi_out, r.phi.data(), r.phi.size() * sizeof(double));
  return r.status;
}

int trstmi_wait(trstmi_server* sv, uint64_t ticket, int timeout_ms, trstmi_result* out,
                double* phi_out) {
  if (!sv || !out) return TRSTMI_EINVAL;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return TRSTMI_ENOTFOUND;
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                         [&] { return sv->reqs[ticket].status != TRSTMI_PENDING; });
  }
  return trstmi_poll(sv, ticket, out, phi_out);
}

int trstmi_cancel(trstmi_server* sv, uint64_t ticket) {
  if (!sv) return TRSTMI_EINVAL;
  std::lock_guard<std::mutex> g(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return TRSTMI_ENOTFOUND;
  if (it->second.status != TRSTMI_PENDING) return it->second.status;
  it->second.cancel = true;
  sv->cv_work.notify_one();
  return TRSTMI_PENDING;
}

int trstmi_server_stats(trstmi_server* sv, trstmi_server_stats_t* out) {
  if (!sv || !out) return TRSTMI_EINVAL;
  std::lock_guard<std::mutex> g(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = sv->submitted;
  out->admitted = sv->admitted;
  out->completed = sv->completed;
  out->cancelled = sv->cancelled;
  out->rounds = sv->rounds;
  out->pairs_scored = sv->pairs_scored;
  out->gpu_busy_s = sv->gpu_busy_s;
  out->hbm_in_use = sv->arena.used();
  out->active_slots = (int32_t)sv->active_count.load();
  out->queued = (int32_t)sv->queue.size();
  out->worker_status = sv->worker_error;
  out->timed_out = sv->timed_out;
  out->kernel_launches = sv->launches.load();
  return TRSTMI_OK;
}

}  // extern "C"
