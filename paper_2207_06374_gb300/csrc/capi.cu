// Host runtime and C ABI of the TRSTMI library (see include/trstmi.h).
//
// One instance = one search: its frame (binary64 master + binary32 copy),
// radius, counters and scratch live in one device allocation.  An iteration
// is a fixed sequence of kernels that read and write the device-resident
// state (DevState), so `iters` iterations are captured once as a CUDA graph
// and replayed with no host round trip; the host synchronises once per call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/trstmi.h"
#include "kernels.h"
#include "trace.h"

using namespace trstmi;

namespace {

constexpr uint32_t kBlobMagic = 0x54525354u;  // "TRST"
constexpr uint32_t kBlobVersion = 1u;
constexpr uint32_t kPairCap = 1u << 16;
// entries of a survivor's pair list (survivor pair pass); a survivor with more
// pairs near its maximum is re-scored over all pairs
constexpr uint32_t kListCap = 4096;
// words zeroed with the top-k scores each iteration: the scores, the list
// counts, the overflow flag and the winner selection (slot, filter needed)
inline size_t top_words(int k) { return 2 * (size_t)k + 3; }
// largest room for the survivors' screen blocks (drawn once per iteration;
// beyond it every tile of the survivor pair pass draws its own two blocks)
constexpr size_t kBlocksMax = (size_t)16 << 20;
constexpr int kGraphChunk = 32;

std::mutex g_attr_mu;
bool g_attr_done[64] = {false};
thread_local char g_last_error[256] = "";

int record_cuda_error(cudaError_t e, const char* what, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (at capi.cu:%d: %.120s)",
                cudaGetErrorName(e), cudaGetErrorString(e), line, what);
  cudaGetLastError();
  return TRSTMI_ECUDA;
}

#define TRY_CUDA(expr)                                             \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return record_cuda_error(_e, #expr, __LINE__); \
  } while (0)

// Validates a device ordinal and prepares it (kernel attributes, once per
// device); the device must already be current (a DeviceGuard holds it).
int ensure_device(int device, int* num_sms) {
  int n = 0;
  TRY_CUDA(cudaGetDeviceCount(&n));
  if (n <= 0) return TRSTMI_ECUDA;
  if (device < 0 || device >= n || device >= 64) return TRSTMI_EINVAL;
  int cur = -1;
  TRY_CUDA(cudaGetDevice(&cur));
  if (cur != device) return TRSTMI_EINVAL;
  {
    std::lock_guard<std::mutex> g(g_attr_mu);
    if (!g_attr_done[device]) {
      TRY_CUDA(init_kernel_attributes());
      g_attr_done[device] = true;
    }
  }
  TRY_CUDA(cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, device));
  return TRSTMI_OK;
}

// The calling thread's current device (the one the stateless entry points use).
int caller_device(int* dev) {
  TRY_CUDA(cudaGetDevice(dev));
  return TRSTMI_OK;
}

// Holds `dev` current for the rest of the enclosing scope (the caller's device
// is restored on return); a device that cannot be made current is an error.
#define USE_DEVICE(dev)                                                         \
  DeviceGuard device_guard_(dev);                                               \
  if (!device_guard_.ok()) {                                                    \
    int n_ = 0;                                                                 \
    if (cudaGetDeviceCount(&n_) != cudaSuccess || n_ < 1) {                     \
      cudaGetLastError();                                                       \
      return TRSTMI_ECUDA;                                                      \
    }                                                                           \
    return TRSTMI_EINVAL;                                                       \
  }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct trstmi_instance {
  int N = 0, d = 0;
  uint64_t seed = 0;
  trstmi_options opt{};
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* block = nullptr;
  size_t block_bytes = 0;
  DeviceMemory dmem;   // where block and the temporary buffers come from
  // carved from block
  DevState* st = nullptr;
  double2* phi64 = nullptr;
  float2* phi32 = nullptr;
  double2* cand64 = nullptr;
  float2* cand32 = nullptr;
  double2* scratch64 = nullptr;
  unsigned int* mu2_k32 = nullptr;         // K
  unsigned long long* mu2_k64 = nullptr;   // K
  unsigned int* mu2_top = nullptr;         // topk, followed by (zeroed with it) the
  uint32_t* scount = nullptr;              // survivor pair lists' counts (topk),
  uint32_t* sover = nullptr;               // a list overflowed (1),
  uint32_t* ssel = nullptr;                // the winner's slot, filter needed (2)
  uint2* slists = nullptr;                 // screen modes: topk x kListCap survivor pairs
  unsigned char* sblocks = nullptr;        // screen modes: the survivors' column blocks in
                                           // the screen layout (when within kBlocksMax)
  uint32_t* topk = nullptr;                // topk
  unsigned int* cert32 = nullptr;          // 1
  unsigned long long* cert64 = nullptr;    // 1
  uint32_t* misc = nullptr;                // [0] npairs, [1] overflow (standalone certify),
                                           // [2] the decide-and-commit launch's CTA counter
  uint2* pairs = nullptr;                  // kPairCap
  TraceRowDev* trace = nullptr;            // trace_cap
  float* planes_top = nullptr;             // screen modes: the top-k survivors drawn once
                                           // for their binary32 re-score (2dN floats each)
  float* planes = nullptr;                 // TRSTMI_FP32: the K candidates of an iteration,
                                           // drawn once as [i][column] planes (2dN floats each)
  std::map<int, cudaGraphExec_t> graphs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_in = nullptr;             // trstmi_set_phi: the caller's frame copied
  DevState* st_host = nullptr;             // pinned host copy of the state (read_state)
  // the device state's screen threshold (infinite when the screen is not
  // used); 0 means every iteration ranks with the screen
  double screen_min_delta = std::numeric_limits<double>::infinity();
};

namespace {

bool is_screen(int p) { return is_screen_precision(p); }

double welch_of(int N, int d) {
  if (N <= d || N < 2) return 0.0;
  return std::sqrt((double)(N - d) / ((double)d * (double)(N - 1)));
}

int cuda_status(cudaError_t e) {
  return e == cudaSuccess ? TRSTMI_OK : record_cuda_error(e, "kernel launch", __LINE__);
}

// binary64 mu^2 of a normalised binary64 frame (with its binary32 rounding)
// into out64: binary32 max, binary32 preselection of the pairs within the
// error bound, binary64 over those pairs, full binary64 pass on overflow.
int enqueue_certify(trstmi_instance* h, const double2* f64, const float2* f32,
                    unsigned long long* out64, const uint32_t* active, uint32_t* npairs,
                    uint32_t* overflow, cudaStream_t s) {
  TRY_CUDA(launch_frame_certify(h->N, h->d, f64, f32, h->cert32, out64, h->pairs, kPairCap,
                                npairs, overflow, active, h->num_sms, s));
  return TRSTMI_OK;
}

__global__ void k_set_mu2cur(DevState* st, const unsigned int* b32, const unsigned long long* b64) {
  st->mu2_cur = b64 ? nonneg_from_bits(*b64) : (double)nonneg_from_bits(*b32);
  st->done = (st->mu2_cur <= st->target2) ? 1u : 0u;
}

__global__ void k_set_stop(DevState* st, uint32_t iters) {
  const unsigned long long stop = (unsigned long long)st->t + iters;
  st->t_stop = stop > 0xffffffffull ? 0xffffffffu : (uint32_t)stop;
  st->t_call = st->t;
  st->accepts_call = st->accepts;
}

// Score the current frame in the deciding precision into st->mu2_cur.
int enqueue_rescore_current(trstmi_instance* h) {
  cudaStream_t s = h->stream;
  const int prec = h->opt.precision;
  if (prec == TRSTMI_FP32) {
    TRY_CUDA(cudaMemsetAsync(h->cert32, 0, 2 * sizeof(unsigned int), s));
    GramSource src{};
    src.perturb = false;
    src.phi = h->phi32;
    TRY_CUDA(launch_gram_f32(h->N, h->d, 1, src, h->cert32, nullptr, h->num_sms, s));
    k_set_mu2cur<<<1, 1, 0, s>>>(h->st, h->cert32, nullptr);
  } else if (prec == TRSTMI_FP64) {
    TRY_CUDA(cudaMemsetAsync(h->cert64, 0, sizeof(unsigned long long), s));
    GramSource src{};
    src.perturb = false;
    src.phi = h->phi64;
    TRY_CUDA(launch_gram_f64(h->N, h->d, 1, src, h->cert64, h->num_sms, s));
    k_set_mu2cur<<<1, 1, 0, s>>>(h->st, nullptr, h->cert64);
  } else {
    // cert32[0..1] and cert64 are one 16-byte span
    TRY_CUDA(cudaMemsetAsync(h->cert32, 0, 2 * sizeof(unsigned int) + sizeof(unsigned long long),
                             s));
    TRY_CUDA(cudaMemsetAsync(h->misc, 0, 2 * sizeof(uint32_t), s));
    int rc = enqueue_certify(h, h->phi64, h->phi32, h->cert64, nullptr, h->misc, h->misc + 1, s);
    if (rc) return rc;
    k_set_mu2cur<<<1, 1, 0, s>>>(h->st, nullptr, h->cert64);
  }
  return cuda_status(cudaGetLastError());
}

// First part of an iteration, enqueued on s: its start (score buffers zeroed,
// whether it runs and how it ranks decided on the device) and the ranking
// scores of candidates c_lo .. c_hi-1 into the K-entry score vector
// (mu2_k64 in binary64, mu2_k32 otherwise).  A whole iteration scores
// 0 .. K-1; a candidate-sharded one scores its rank's range.
int enqueue_iteration_score(trstmi_instance* h, cudaStream_t s, int c_lo, int c_hi,
                            uint32_t call_iters = 0) {
  const int N = h->N, d = h->d, K = h->opt.K;
  const int count = c_hi - c_lo;
  DevState* st = h->st;
  const int prec = h->opt.precision;
  if (prec == TRSTMI_FP64) {
    TRY_CUDA(launch_iter_begin(st, h->mu2_k64, sizeof(unsigned long long) * K, nullptr, 0,
                               nullptr, 0, s, call_iters));
    if (count > 0) {
      GramSource src{};
      src.perturb = true;
      src.phi = h->phi64;
      src.seed = h->seed;
      src.c0 = (uint32_t)c_lo;
      src.st = st;
      TRY_CUDA(launch_gram_f64(N, d, count, src, h->mu2_k64 + c_lo, h->num_sms, s));
    }
  } else if (prec == TRSTMI_FP32) {
    TRY_CUDA(launch_iter_begin(st, h->mu2_k32, sizeof(unsigned int) * K, nullptr, 0, nullptr,
                               0, s, call_iters));
    if (count > 0) {
      GramSource src{};
      src.perturb = true;
      src.phi = h->phi32;
      src.seed = h->seed;
      src.c0 = (uint32_t)c_lo;
      src.st = st;
      if (h->planes) {
        TRY_CUDA(launch_gen_planes_f32(N, d, count, h->phi32, h->seed, (uint32_t)c_lo, st, 0u,
                                       0.0, h->planes, s));
        src.planes = h->planes;
      }
      TRY_CUDA(launch_gram_f32(N, d, count, src, h->mu2_k32 + c_lo, nullptr, h->num_sms, s));
    }
  } else {
    const int k = h->opt.topk;
    TRY_CUDA(launch_iter_begin(st, h->mu2_k32, sizeof(unsigned int) * K, h->mu2_top,
                               top_words(k) * sizeof(uint32_t), h->cert32,
                               2 * sizeof(unsigned int) + sizeof(unsigned long long), s,
                               call_iters));
    if (count > 0) {
      // rank the candidates: tensor-core screen while delta >= screen_min_delta,
      // else the fp32 Gram of every candidate (each kernel returns at once when
      // the other one is selected for this iteration)
      if (screen_supported(N, d, screen_fmt_of(prec, d)))
        TRY_CUDA(launch_screen(screen_fmt_of(prec, d), N, d, h->seed, h->phi32, count,
                               (uint32_t)c_lo, 0u, 0.0, st, h->mu2_k32 + c_lo, &st->error,
                               h->num_sms, s));
      // (not enqueued at all when every iteration screens)
      if (!(h->screen_min_delta <= 0.0)) {
        GramSource full{};
        full.perturb = true;
        full.phi = h->phi32;
        full.seed = h->seed;
        full.c0 = (uint32_t)c_lo;
        full.st = st;
        full.gate = &st->use_full;
        TRY_CUDA(launch_gram_f32(N, d, count, full, h->mu2_k32 + c_lo, nullptr, h->num_sms, s));
      }
    }
  }
  return TRSTMI_OK;
}

// Second part: selection from the full score vector, and in the screen modes
// the fp32 re-score of the top-k and the binary64 certification of the best
// survivor; then the accept/radius rule, the trace row and the commit.
int enqueue_iteration_finish(trstmi_instance* h, cudaStream_t s) {
  const int N = h->N, d = h->d, K = h->opt.K;
  DevState* st = h->st;
  const int prec = h->opt.precision;
  if (prec == TRSTMI_FP64) {
    TRY_CUDA(launch_select_decide_f64(st, h->mu2_k64, K, h->trace, s));
    TRY_CUDA(launch_commit_f64(N, d, h->seed, st, h->phi64, h->phi32, s));
  } else if (prec == TRSTMI_FP32) {
    TRY_CUDA(launch_select_decide_f32(st, h->mu2_k32, K, h->trace, s));
    TRY_CUDA(launch_commit_f32(N, d, h->seed, st, h->phi32, h->phi64, s));
  } else {
    const int k = h->opt.topk;
    const int fmt = screen_fmt_of(prec, d);
    const bool screens = screen_supported(N, d, fmt);
    // an iteration that ranked with the binary32 Gram of every candidate
    // certifies through the binary32 filter pass; none does when every
    // iteration screens
    const bool filter = !(h->screen_min_delta <= 0.0);
    TRY_CUDA(launch_topk(st, h->mu2_k32, K, k, h->topk, h->mu2_top, s));
    // the survivors' re-score in binary32 when the screen ranked them (else
    // k_topk copied the binary32 scores of the full ranking pass): over the
    // pairs the survivor pair pass lists (every pair that can be a survivor's
    // binary32 or binary64 maximum), each pair's two columns drawn with the
    // bits of the survivors' draw; only when a list overflowed, the survivors
    // drawn whole (the tile pass's gen_column arithmetic) and re-scored over
    // all pairs
    GramSource src{};
    src.perturb = true;
    src.phi = h->phi32;
    src.seed = h->seed;
    src.cand_list = h->topk;
    src.st = st;
    src.planes = h->planes_top;
    const uint32_t* full_gate = &st->use_screen;
    if (screens) {
      TRY_CUDA(launch_screen_pairs(fmt, N, d, h->seed, h->phi32, st, h->topk, h->mu2_k32, k,
                                   screen_pair_err(fmt), h->slists, h->scount, kListCap, h->sover,
                                   &st->error, h->num_sms, s, h->sblocks));
      TRY_CUDA(launch_pairs32(st, h->slists, h->scount, kListCap, k, N, d, h->phi32, h->seed,
                              h->topk, h->mu2_top, s));
      full_gate = h->sover;
    }
    src.gate = full_gate;
    TRY_CUDA(launch_gen_planes_f32(N, d, k, h->phi32, h->seed, 0u, st, 0u, 0.0, h->planes_top, s,
                                   h->topk, full_gate));
    TRY_CUDA(launch_gram_f32(N, d, k, src, h->mu2_top, nullptr, h->num_sms, s));
    TRY_CUDA(launch_materialize64(N, d, h->seed, st, h->topk, h->mu2_top, k, h->phi64,
                                  h->cand64, h->cand32, s, h->cert32, h->scount,
                                  screens ? kListCap : 0u, h->ssel, filter));
    // certification of a survivor the rule could accept (st->certify):
    // binary64 over the winner's listed pairs, or over the pairs the binary32
    // filter pass keeps from the survivor's binary32 score as the hint
    // (cert32[0..1] and cert64 were zeroed by iter_begin), or over all pairs
    // when neither covers the maximum (st->overflow)
    if (filter) {
      GramSource fs{};
      fs.perturb = false;
      fs.phi = h->cand32;
      fs.normalize = false;
      fs.gate = &h->ssel[1];
      PairFilter pf{h->cert32, certify_margin(d), h->pairs, &st->npairs, kPairCap, &st->overflow,
                    nullptr, (float)certify_margin_mu2(d)};
      TRY_CUDA(launch_gram_f32(N, d, 1, fs, h->cert32 + 1, &pf, h->num_sms, s));
    }
    TRY_CUDA(launch_pairs64(&st->certify, &st->npairs, h->pairs, kPairCap, d, h->cand64,
                            h->cert64, s, h->cert32, h->cert32 + 1,
                            (float)certify_margin_mu2(d), &st->overflow, h->ssel, h->slists,
                            h->scount, screens ? kListCap : 0u));
    GramSource full{};
    full.perturb = false;
    full.phi = h->cand64;
    full.normalize = false;
    full.gate = &st->overflow;  // reset every iteration, so 0 when the iteration is inactive
    TRY_CUDA(launch_gram_f64(N, d, 1, full, h->cert64, h->num_sms, s));
    TRY_CUDA(launch_decide_commit(N, d, st, h->cert64, h->trace, h->cand64, h->cand32,
                                  h->phi64, h->phi32, &h->misc[2], s));
  }
  return TRSTMI_OK;
}

// One iteration of the search, enqueued on s (captured into the graph).
int enqueue_iteration(trstmi_instance* h, cudaStream_t s, uint32_t call_iters = 0) {
  const int rc = enqueue_iteration_score(h, s, 0, h->opt.K, call_iters);
  return rc ? rc : enqueue_iteration_finish(h, s);
}

// The graph of `iters` iterations; with_stop: it is a whole trstmi_step call,
// and its first kernel also sets the call's stop and start counters.
int get_graph(trstmi_instance* h, int iters, cudaGraphExec_t* out, bool with_stop = false) {
  const int key = 2 * iters + (with_stop ? 1 : 0);
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) { *out = it->second; return TRSTMI_OK; }
  cudaGraph_t g = nullptr;
  TRY_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = TRSTMI_OK;
  for (int i = 0; i < iters && rc == TRSTMI_OK; ++i)
    rc = enqueue_iteration(h, h->stream, (with_stop && i == 0) ? (uint32_t)iters : 0u);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (rc != TRSTMI_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != TRSTMI_OK ? rc : TRSTMI_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return TRSTMI_ECUDA;
  h->graphs[key] = ex;
  *out = ex;
  return TRSTMI_OK;
}

// The device state, through a pinned host copy (a direct copy, not staged).
int read_state(trstmi_instance* h, DevState* out) {
  TRY_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                           h->stream));
  TRY_CUDA(cudaStreamSynchronize(h->stream));
  *out = *h->st_host;
  return TRSTMI_OK;
}

int device_error_status(const DevState& s) {
  if (s.error & kErrTimeout) return TRSTMI_ETIMEOUT;
  if (s.error & kErrZeroColumn) return TRSTMI_EINVAL;
  return TRSTMI_OK;
}

int validate_options(int N, int d, const trstmi_options& o) {
  if (N < 2 || d < 1 || d > kMaxD) return TRSTMI_EINVAL;
  if ((long long)N * ((d + 1) / 2) >= (1ll << 32)) return TRSTMI_EINVAL;
  if (o.K < 1 || o.trace_cap < 0) return TRSTMI_EINVAL;
  if (o.precision < TRSTMI_FP64 || o.precision > TRSTMI_TF32_SCREEN) return TRSTMI_EINVAL;
  if (is_screen(o.precision) && (o.topk < 1 || o.topk > 64 || o.topk > o.K))
    return TRSTMI_EINVAL;
  if (!(o.delta0 > 0) || !(o.gamma_inc >= 1) || !(o.gamma_dec > 0 && o.gamma_dec <= 1))
    return TRSTMI_EINVAL;
  if (!(o.delta_min >= 0) || !(o.delta_max >= o.delta_min)) return TRSTMI_EINVAL;
  if (!(o.screen_min_delta >= 0)) return TRSTMI_EINVAL;
  if (!DeviceMemory::valid(o)) return TRSTMI_EINVAL;
  return TRSTMI_OK;
}

}  // namespace

extern "C" {

void trstmi_default_options(trstmi_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->K = 256;
  o->precision = TRSTMI_FP64;
  o->topk = 8;
  o->trace_cap = 4096;
  o->delta0 = 0.1;
  o->gamma_inc = 2.0;
  o->gamma_dec = 0.25;
  o->delta_min = 1e-9;
  o->delta_max = 1.0;
  o->target_mu = 0.0;
  o->screen_min_delta = 0.01;
  o->stream = nullptr;
  o->device = 0;
}

const char* trstmi_last_error(void) { return g_last_error; }

const char* trstmi_strerror(int s) {
  switch (s) {
    case TRSTMI_OK: return "ok";
    case TRSTMI_PENDING: return "pending";
    case TRSTMI_EINVAL: return "invalid argument";
    case TRSTMI_ENOMEM: return "out of device memory or over budget";
    case TRSTMI_ECUDA: return "CUDA error or no CUDA device";
    case TRSTMI_ETIMEOUT: return "device-side wait timed out";
    case TRSTMI_ECANCELLED: return "cancelled";
    case TRSTMI_EBUSY: return "queue full";
    case TRSTMI_EUNSUPPORTED: return "shape/precision combination not supported";
    case TRSTMI_ENOTFOUND: return "unknown ticket";
    case TRSTMI_ESIZE: return "size beyond the built-in limit of this entry point";
    default: return "unknown status";
  }
}

void trstmi_destroy(trstmi_handle h) {
  if (!h) return;
  DeviceGuard device_guard(h->opt.device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->st_host) cudaFreeHost(h->st_host);
  h->dmem.release(h->block);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int trstmi_create(int N, int d, uint64_t seed, const trstmi_options* opt, trstmi_handle* out) {
  trstmi::TraceRange trace_range("trstmi_create");
  if (!out) return TRSTMI_EINVAL;
  *out = nullptr;
  trstmi_options o;
  if (opt) o = *opt; else trstmi_default_options(&o);
  if (!is_screen(o.precision)) o.topk = std::max(1, std::min(o.topk, o.K));
  int num_sms = 0;
  int rc = validate_options(N, d, o);
  if (rc) return rc;
  USE_DEVICE(o.device);
  rc = ensure_device(o.device, &num_sms);
  if (rc) return rc;

  trstmi_instance* h = new (std::nothrow) trstmi_instance();
  if (!h) return TRSTMI_ENOMEM;
  h->N = N; h->d = d; h->seed = seed; h->opt = o; h->num_sms = num_sms;
  h->dmem = DeviceMemory(o);
  if (o.stream) {
    h->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return TRSTMI_ECUDA;
    }
    h->own_stream = true;
  }
  // carve one allocation
  const size_t nd = (size_t)N * d;
  const int K = o.K, k = std::max(1, o.topk);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes, 256); return at; };
  const size_t o_st = take(sizeof(DevState));
  const size_t o_phi64 = take(nd * sizeof(double2));
  const size_t o_phi32 = take(nd * sizeof(float2));
  const size_t o_c64 = take(nd * sizeof(double2));
  const size_t o_c32 = take(nd * sizeof(float2));
  const size_t o_s64 = take(nd * sizeof(double2));
  const size_t o_k32 = take((size_t)K * sizeof(unsigned int));
  const size_t o_k64 = take((size_t)K * sizeof(unsigned long long));
  const size_t o_top = take(top_words(k) * sizeof(uint32_t));
  const size_t o_topk = take((size_t)k * sizeof(uint32_t));
  // cert32[2] followed by cert64 in one 16-byte span (zeroed together)
  const size_t o_cert = take(2 * sizeof(unsigned int) + sizeof(unsigned long long));
  const size_t o_misc = take(4 * sizeof(uint32_t));
  const size_t o_pairs = take((size_t)kPairCap * sizeof(uint2));
  const size_t o_trace = take((size_t)std::max(o.trace_cap, 1) * sizeof(TraceRowDev));
  // TRSTMI_FP32: room for the iteration's K candidates (up to 1 GiB), so each
  // is drawn once and its tiles read it, instead of every tile redrawing its
  // two column blocks
  const size_t planes_bytes = (size_t)K * 2 * nd * sizeof(float);
  const size_t o_planes = (o.precision == TRSTMI_FP32 && planes_bytes <= ((size_t)1 << 30))
                              ? take(planes_bytes) : (size_t)-1;
  const size_t o_ptop = is_screen(o.precision) ? take((size_t)k * 2 * nd * sizeof(float))
                                               : (size_t)-1;
  const size_t o_lists = is_screen(o.precision) ? take((size_t)k * kListCap * sizeof(uint2))
                                                : (size_t)-1;
  const int sfmt = screen_fmt_of(o.precision, d);
  const size_t blocks_bytes = is_screen(o.precision) && screen_supported(N, d, sfmt)
                                  ? (size_t)k * ((N + 127) / 128) * screen_block_bytes(sfmt)
                                  : 0;
  const size_t o_blocks = (blocks_bytes > 0 && blocks_bytes <= kBlocksMax) ? take(blocks_bytes)
                                                                          : (size_t)-1;
  h->block_bytes = off;
  if (h->dmem.allocate(&h->block, off) != cudaSuccess) {
    cudaGetLastError();
    trstmi_destroy(h);
    return TRSTMI_ENOMEM;
  }
  char* b = (char*)h->block;
  h->st = (DevState*)(b + o_st);
  h->phi64 = (double2*)(b + o_phi64);
  h->phi32 = (float2*)(b + o_phi32);
  h->cand64 = (double2*)(b + o_c64);
  h->cand32 = (float2*)(b + o_c32);
  h->scratch64 = (double2*)(b + o_s64);
  h->mu2_k32 = (unsigned int*)(b + o_k32);
  h->mu2_k64 = (unsigned long long*)(b + o_k64);
  h->mu2_top = (unsigned int*)(b + o_top);
  h->scount = (uint32_t*)(b + o_top) + k;
  h->sover = h->scount + k;
  h->ssel = h->sover + 1;
  h->topk = (uint32_t*)(b + o_topk);
  h->cert32 = (unsigned int*)(b + o_cert);
  h->cert64 = (unsigned long long*)(b + o_cert + 2 * sizeof(unsigned int));
  h->misc = (uint32_t*)(b + o_misc);
  h->pairs = (uint2*)(b + o_pairs);
  h->trace = (TraceRowDev*)(b + o_trace);
  if (o_planes != (size_t)-1) h->planes = (float*)(b + o_planes);
  if (o_ptop != (size_t)-1) h->planes_top = (float*)(b + o_ptop);
  if (o_lists != (size_t)-1) h->slists = (uint2*)(b + o_lists);
  if (o_blocks != (size_t)-1) h->sblocks = (unsigned char*)(b + o_blocks);
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&h->st_host, sizeof(DevState)) != cudaSuccess) {
    trstmi_destroy(h);
    return TRSTMI_ECUDA;
  }
  DevState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.delta = o.delta0;
  s0.delta_used = o.delta0;
  s0.target2 = o.target_mu > 0 ? o.target_mu * o.target_mu : -1.0;
  s0.gamma_inc = o.gamma_inc;
  s0.gamma_dec = o.gamma_dec;
  s0.delta_min = o.delta_min;
  s0.delta_max = o.delta_max;
  // a shape outside the screen kernel's range ranks with the binary32 Gram,
  // and the plain modes never use the screen (trace flag bit 0 stays clear)
  s0.screen_min_delta = (!is_screen(o.precision) ||
                         !screen_supported(N, d, screen_fmt_of(o.precision, d)))
                            ? std::numeric_limits<double>::infinity()
                            : o.screen_min_delta;
  s0.trace_cap = (uint32_t)o.trace_cap;
  h->screen_min_delta = s0.screen_min_delta;
  cudaStream_t s = h->stream;
  if (cudaMemsetAsync(h->block, 0, off, s) != cudaSuccess ||
      cudaMemcpyAsync(h->st, &s0, sizeof(s0), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      launch_init_frame(N, d, seed, h->phi64, h->phi32, h->st, s) != cudaSuccess) {
    trstmi_destroy(h);
    return TRSTMI_ECUDA;
  }
  rc = enqueue_rescore_current(h);
  DevState chk;
  if (!rc) rc = read_state(h, &chk);
  if (!rc) rc = device_error_status(chk);
  if (rc) { trstmi_destroy(h); return rc; }
  *out = h;
  return TRSTMI_OK;
}

int trstmi_step(trstmi_handle h, int iters, trstmi_step_info* info) {
  trstmi::TraceRange trace_range("trstmi_step");
  if (!h || iters < 0) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  // graphs are captured (host work only) before the timed span starts
  const int full = iters / kGraphChunk, rem = iters % kGraphChunk;
  // a call of fewer than kGraphChunk iterations is one graph whose first
  // kernel sets the call's stop; longer calls set it in a kernel of their own
  const bool whole = full == 0 && rem > 0;
  cudaGraphExec_t g_full = nullptr, g_rem = nullptr;
  int rc = TRSTMI_OK;
  if (full > 0 && (rc = get_graph(h, kGraphChunk, &g_full)) != TRSTMI_OK) return rc;
  if (rem > 0 && (rc = get_graph(h, rem, &g_rem, whole)) != TRSTMI_OK) return rc;
  // no host synchronisation until the end: the start counters are snapshot
  // on the device by the first kernel
  TRY_CUDA(cudaEventRecord(h->ev0, s));
  if (!whole) {
    k_set_stop<<<1, 1, 0, s>>>(h->st, (uint32_t)iters);
    TRY_CUDA(cudaGetLastError());
  }
  for (int r = 0; r < full; ++r) TRY_CUDA(cudaGraphLaunch(g_full, s));
  if (g_rem) TRY_CUDA(cudaGraphLaunch(g_rem, s));
  TRY_CUDA(cudaEventRecord(h->ev1, s));
  DevState after;
  rc = read_state(h, &after);
  if (rc) return rc;
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->iters_done = (int32_t)(after.t - after.t_call);
    info->accepts = (int32_t)(after.accepts - after.accepts_call);
    info->mu = std::sqrt(after.mu2_cur);
    info->delta = after.delta;
    info->pairs_scored = (uint64_t)info->iters_done * (uint64_t)h->opt.K *
                         ((uint64_t)h->N * (uint64_t)(h->N - 1) / 2);
    info->elapsed_ns = (uint64_t)((double)ms * 1e6);
    info->done = (int32_t)after.done;
    info->reserved = 0;
  }
  return device_error_status(after);
}

int trstmi_shard_score_bytes(trstmi_handle h, size_t* bytes) {
  if (!h || !bytes) return TRSTMI_EINVAL;
  *bytes = (size_t)h->opt.K *
           (h->opt.precision == TRSTMI_FP64 ? sizeof(unsigned long long) : sizeof(unsigned int));
  return TRSTMI_OK;
}

int trstmi_shard_score(trstmi_handle h, int c_lo, int c_hi, void* scores) {
  trstmi::TraceRange trace_range("trstmi_shard_score");
  if (!h || !scores || c_lo < 0 || c_hi < c_lo || c_hi > h->opt.K) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  k_set_stop<<<1, 1, 0, s>>>(h->st, 1u);
  TRY_CUDA(cudaGetLastError());
  int rc = enqueue_iteration_score(h, s, c_lo, c_hi);
  if (rc) return rc;
  const bool f64 = h->opt.precision == TRSTMI_FP64;
  size_t bytes = 0;
  trstmi_shard_score_bytes(h, &bytes);
  TRY_CUDA(cudaMemcpyAsync(scores, f64 ? (const void*)h->mu2_k64 : (const void*)h->mu2_k32, bytes,
                           cudaMemcpyDeviceToDevice, s));
  if (h->own_stream) TRY_CUDA(cudaStreamSynchronize(s));
  return TRSTMI_OK;
}

int trstmi_shard_finish(trstmi_handle h, const void* scores, trstmi_step_info* info) {
  trstmi::TraceRange trace_range("trstmi_shard_finish");
  if (!h || !scores) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  const bool f64 = h->opt.precision == TRSTMI_FP64;
  size_t bytes = 0;
  trstmi_shard_score_bytes(h, &bytes);
  TRY_CUDA(cudaEventRecord(h->ev0, s));
  TRY_CUDA(cudaMemcpyAsync(f64 ? (void*)h->mu2_k64 : (void*)h->mu2_k32, scores, bytes,
                           cudaMemcpyDeviceToDevice, s));
  int rc = enqueue_iteration_finish(h, s);
  if (rc) return rc;
  TRY_CUDA(cudaEventRecord(h->ev1, s));
  DevState after;
  rc = read_state(h, &after);
  if (rc) return rc;
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->iters_done = (int32_t)(after.t - after.t_call);
    info->accepts = (int32_t)(after.accepts - after.accepts_call);
    info->mu = std::sqrt(after.mu2_cur);
    info->delta = after.delta;
    info->pairs_scored = (uint64_t)info->iters_done * (uint64_t)h->opt.K *
                         ((uint64_t)h->N * (uint64_t)(h->N - 1) / 2);
    info->elapsed_ns = (uint64_t)((double)ms * 1e6);
    info->done = (int32_t)after.done;
    info->reserved = 0;
  }
  return device_error_status(after);
}

int trstmi_coherence(trstmi_handle h, double* mu, double* welch) {
  if (!h || !mu) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  TRY_CUDA(cudaMemsetAsync(h->cert32, 0, 2 * sizeof(unsigned int) + sizeof(unsigned long long), s));
  TRY_CUDA(cudaMemsetAsync(h->misc, 0, 2 * sizeof(uint32_t), s));
  TRY_CUDA(launch_normalize64(h->N, h->d, h->phi64, h->scratch64, h->cand32, nullptr, s));
  int rc = enqueue_certify(h, h->scratch64, h->cand32, h->cert64, nullptr, h->misc, h->misc + 1, s);
  if (rc) return rc;
  unsigned long long bits = 0;
  TRY_CUDA(cudaMemcpyAsync(&bits, h->cert64, sizeof(bits), cudaMemcpyDeviceToHost, s));
  TRY_CUDA(cudaStreamSynchronize(s));
  double m2;
  std::memcpy(&m2, &bits, sizeof(m2));
  *mu = std::sqrt(m2);
  if (welch) *welch = welch_of(h->N, h->d);
  return TRSTMI_OK;
}

int trstmi_get_phi(trstmi_handle h, double* out) {
  if (!h || !out) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  TRY_CUDA(cudaMemcpyAsync(out, h->phi64, (size_t)h->N * h->d * sizeof(double2),
                           cudaMemcpyDeviceToHost, h->stream));
  TRY_CUDA(cudaStreamSynchronize(h->stream));
  return TRSTMI_OK;
}

int trstmi_set_phi(trstmi_handle h, const double* in) {
  if (!h || !in) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  const size_t bytes = (size_t)h->N * h->d * sizeof(double2);
  // the copy into scratch (not yet the frame) runs while the host checks the
  // columns; the caller's buffer is read only until ev_in
  TRY_CUDA(cudaMemcpyAsync(h->scratch64, in, bytes, cudaMemcpyHostToDevice, s));
  TRY_CUDA(cudaEventRecord(h->ev_in, s));
  // reject zero or non-finite columns before the device state changes; four
  // partial sums per column keep the check off one long chain of dependent
  // additions (a sum of squares is zero exactly when every entry is)
  const int m = 2 * h->d;
  bool ok = true;
  for (int j = 0; j < h->N && ok; ++j) {
    const double* c = in + (size_t)j * m;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = 0;
    for (; i + 4 <= m; i += 4) {
      a0 += c[i] * c[i];
      a1 += c[i + 1] * c[i + 1];
      a2 += c[i + 2] * c[i + 2];
      a3 += c[i + 3] * c[i + 3];
    }
    for (; i < m; ++i) a0 += c[i] * c[i];
    const double acc = (a0 + a1) + (a2 + a3);
    ok = acc > 0.0 && std::isfinite(acc);
  }
  if (!ok) {
    TRY_CUDA(cudaEventSynchronize(h->ev_in));
    return TRSTMI_EINVAL;
  }
  // renormalise into the frame and rescore, in stream order before any later
  // call's work; return once the caller's buffer has been read
  TRY_CUDA(launch_normalize64(h->N, h->d, h->scratch64, h->phi64, h->phi32, h->st, s));
  const int rc = enqueue_rescore_current(h);
  TRY_CUDA(cudaEventSynchronize(h->ev_in));
  return rc;
}

namespace {
struct BlobHeader {
  uint32_t magic, version;
  int32_t N, d;
  uint64_t seed;
  int32_t precision, K, topk, pad;
  DevState st;
};
}  // namespace

int trstmi_get_state(trstmi_handle h, void* blob, size_t* size) {
  if (!h || !size) return TRSTMI_EINVAL;
  const size_t nd = (size_t)h->N * h->d;
  const size_t need = sizeof(BlobHeader) + nd * sizeof(double2) + nd * sizeof(float2);
  if (!blob) { *size = need; return TRSTMI_OK; }
  if (*size < need) { *size = need; return TRSTMI_EINVAL; }
  USE_DEVICE(h->opt.device);
  BlobHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  hd.magic = kBlobMagic; hd.version = kBlobVersion; hd.N = h->N; hd.d = h->d; hd.seed = h->seed;
  hd.precision = h->opt.precision; hd.K = h->opt.K; hd.topk = h->opt.topk;
  char* p = (char*)blob;
  TRY_CUDA(cudaMemcpyAsync(&hd.st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  TRY_CUDA(cudaMemcpyAsync(p + sizeof(BlobHeader), h->phi64, nd * sizeof(double2),
                           cudaMemcpyDeviceToHost, h->stream));
  TRY_CUDA(cudaMemcpyAsync(p + sizeof(BlobHeader) + nd * sizeof(double2), h->phi32,
                           nd * sizeof(float2), cudaMemcpyDeviceToHost, h->stream));
  TRY_CUDA(cudaStreamSynchronize(h->stream));
  std::memcpy(p, &hd, sizeof(hd));
  *size = need;
  return TRSTMI_OK;
}

int trstmi_set_state(trstmi_handle h, const void* blob, size_t size) {
  if (!h || !blob || size < sizeof(BlobHeader)) return TRSTMI_EINVAL;
  BlobHeader hd;
  std::memcpy(&hd, blob, sizeof(hd));
  const size_t nd = (size_t)h->N * h->d;
  if (hd.magic != kBlobMagic || hd.version != kBlobVersion || hd.N != h->N || hd.d != h->d ||
      hd.seed != h->seed || hd.precision != h->opt.precision || hd.K != h->opt.K ||
      size < sizeof(BlobHeader) + nd * (sizeof(double2) + sizeof(float2)))
    return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  DevState st = hd.st;
  st.trace_cap = (uint32_t)h->opt.trace_cap;
  st.screen_min_delta = h->screen_min_delta;   // this handle's options rule
  const char* p = (const char*)blob;
  TRY_CUDA(cudaMemcpyAsync(h->st, &st, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  TRY_CUDA(cudaMemcpyAsync(h->phi64, p + sizeof(BlobHeader), nd * sizeof(double2),
                           cudaMemcpyHostToDevice, h->stream));
  TRY_CUDA(cudaMemcpyAsync(h->phi32, p + sizeof(BlobHeader) + nd * sizeof(double2),
                           nd * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
  TRY_CUDA(cudaStreamSynchronize(h->stream));
  return TRSTMI_OK;
}

int trstmi_get_trace(trstmi_handle h, trstmi_trace_row* rows, int n, int* n_out) {
  if (!h || n < 0 || !n_out || (n > 0 && !rows)) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  static_assert(sizeof(trstmi_trace_row) == sizeof(TraceRowDev), "trace row layout");
  DevState s;
  int rc = read_state(h, &s);
  if (rc) return rc;
  const uint32_t cap = s.trace_cap;
  const uint32_t avail = std::min<uint32_t>(cap, s.t);
  const uint32_t cnt = std::min<uint32_t>(avail, (uint32_t)n);
  std::vector<TraceRowDev> all(cap ? cap : 1);
  if (cap) {
    TRY_CUDA(cudaMemcpyAsync(all.data(), h->trace, cap * sizeof(TraceRowDev),
                             cudaMemcpyDeviceToHost, h->stream));
    TRY_CUDA(cudaStreamSynchronize(h->stream));
  }
  for (uint32_t q = 0; q < cnt; ++q) {
    const uint32_t t = s.t - cnt + 1 + q;  // 1-based iteration
    std::memcpy(&rows[q], &all[(t - 1) % cap], sizeof(TraceRowDev));
  }
  *n_out = (int)cnt;
  return TRSTMI_OK;
}

int trstmi_score(trstmi_handle h, uint32_t t, uint32_t c0, int count, double delta,
                 int precision, double* mu2) {
  if (!h || count < 0 || (count > 0 && !mu2) || t < 1 || !(delta >= 0)) return TRSTMI_EINVAL;
  if (count == 0) return TRSTMI_OK;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  void* tmp = nullptr;
  const size_t bytes = (size_t)count * sizeof(unsigned long long);
  TRY_CUDA(h->dmem.allocate(&tmp, bytes));
  int rc = TRSTMI_OK;
  std::vector<double> outv(count);
  do {
    if (cudaMemsetAsync(tmp, 0, bytes, s) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    GramSource src{};
    src.perturb = true;
    src.seed = h->seed;
    src.c0 = c0;
    src.t = t;
    src.delta = delta;
    if (precision == TRSTMI_FP64) {
      src.phi = h->phi64;
      if (launch_gram_f64(h->N, h->d, count, src, (unsigned long long*)tmp, h->num_sms, s)) {
        rc = TRSTMI_ECUDA; break;
      }
      std::vector<unsigned long long> b(count);
      if (cudaMemcpyAsync(b.data(), tmp, bytes, cudaMemcpyDeviceToHost, s) ||
          cudaStreamSynchronize(s)) { rc = TRSTMI_ECUDA; break; }
      for (int q = 0; q < count; ++q) std::memcpy(&outv[q], &b[q], sizeof(double));
    } else if (precision == TRSTMI_FP32 || is_screen(precision)) {
      cudaError_t e;
      if (precision == TRSTMI_FP32) {
        src.phi = h->phi32;
        e = launch_gram_f32(h->N, h->d, count, src, (unsigned int*)tmp, nullptr, h->num_sms, s);
      } else {
        if (!screen_supported(h->N, h->d, screen_fmt_of(precision, h->d))) { rc = TRSTMI_EUNSUPPORTED; break; }
        e = cudaMemsetAsync(&h->misc[1], 0, sizeof(uint32_t), s);
        if (e == cudaSuccess)
          e = launch_screen(screen_fmt_of(precision, h->d), h->N, h->d, h->seed, h->phi32, count,
                            c0, t, delta, nullptr, (unsigned int*)tmp, &h->misc[1], h->num_sms, s);
      }
      if (e != cudaSuccess) { rc = record_cuda_error(e, "score kernel launch", __LINE__); break; }
      std::vector<unsigned int> b(count);
      uint32_t err = 0;
      if (cudaMemcpyAsync(b.data(), tmp, (size_t)count * sizeof(unsigned int),
                          cudaMemcpyDeviceToHost, s) ||
          (precision != TRSTMI_FP32 &&
           cudaMemcpyAsync(&err, &h->misc[1], sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) ||
          cudaStreamSynchronize(s)) { rc = TRSTMI_ECUDA; break; }
      if (err & kErrTimeout) { rc = TRSTMI_ETIMEOUT; break; }
      for (int q = 0; q < count; ++q) {
        float f;
        std::memcpy(&f, &b[q], sizeof(float));
        outv[q] = (double)f;
      }
    } else {
      rc = TRSTMI_EINVAL;
    }
  } while (0);
  cudaStreamSynchronize(s);   // the buffer is released only once the stream is done with it
  h->dmem.release(tmp);
  if (rc == TRSTMI_OK) std::memcpy(mu2, outv.data(), sizeof(double) * count);
  return rc;
}

int trstmi_last_ranking(trstmi_handle h, double* mu2, uint32_t* survivors,
                        double* mu2_survivors) {
  if (!h) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  const int K = h->opt.K, k = h->opt.topk;
  const bool f64 = h->opt.precision == TRSTMI_FP64;
  const bool screen = is_screen(h->opt.precision);
  if ((survivors || mu2_survivors) && !screen) return TRSTMI_EINVAL;
  cudaStream_t s = h->stream;
  std::vector<unsigned long long> b64(f64 ? K : 0);
  std::vector<unsigned int> b32(f64 ? 0 : K), t32(screen ? k : 0);
  std::vector<uint32_t> idx(screen ? k : 0);
  if (mu2) {
    if (f64) TRY_CUDA(cudaMemcpyAsync(b64.data(), h->mu2_k64, K * sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, s));
    else TRY_CUDA(cudaMemcpyAsync(b32.data(), h->mu2_k32, K * sizeof(unsigned int),
                                  cudaMemcpyDeviceToHost, s));
  }
  if (screen) {
    TRY_CUDA(cudaMemcpyAsync(idx.data(), h->topk, k * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaMemcpyAsync(t32.data(), h->mu2_top, k * sizeof(unsigned int),
                             cudaMemcpyDeviceToHost, s));
  }
  TRY_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; mu2 && c < K; ++c) {
    if (f64) {
      std::memcpy(&mu2[c], &b64[c], sizeof(double));
    } else {
      float f;
      std::memcpy(&f, &b32[c], sizeof(float));
      mu2[c] = (double)f;
    }
  }
  for (int q = 0; q < k && screen; ++q) {
    if (survivors) survivors[q] = idx[q];
    if (mu2_survivors) {
      float f;
      std::memcpy(&f, &t32[q], sizeof(float));
      mu2_survivors[q] = (double)f;
    }
  }
  return TRSTMI_OK;
}

int trstmi_candidate(trstmi_handle h, uint32_t t, uint32_t c, double delta, int precision,
                     double* out) {
  if (!h || !out || t < 1 || !(delta >= 0)) return TRSTMI_EINVAL;
  if (precision != TRSTMI_FP64 && precision != TRSTMI_FP32) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  TRY_CUDA(launch_gen_candidate(h->N, h->d, h->seed, t, c, delta, precision == TRSTMI_FP64,
                                h->phi64, h->phi32, h->scratch64, s));
  TRY_CUDA(cudaMemcpyAsync(out, h->scratch64, (size_t)h->N * h->d * sizeof(double2),
                           cudaMemcpyDeviceToHost, s));
  TRY_CUDA(cudaStreamSynchronize(s));
  return TRSTMI_OK;
}

int trstmi_mu2_frame(int N, int d, const double* phi, int precision, double* mu2) {
  if (N < 1 || d < 1 || d > kMaxD || !phi || !mu2) return TRSTMI_EINVAL;
  if (precision != TRSTMI_FP64 && precision != TRSTMI_FP32) return TRSTMI_EINVAL;
  int num_sms = 0, dev = 0;
  int rc = caller_device(&dev);
  if (rc || (rc = ensure_device(dev, &num_sms)) != TRSTMI_OK) return rc;
  const size_t nd = (size_t)N * d;
  void* buf = nullptr;
  const size_t bytes = nd * sizeof(double2) + 256;
  TRY_CUDA(cudaMalloc(&buf, bytes));
  std::vector<float> f32;
  do {
    GramSource src{};
    src.perturb = false;
    src.phi = (char*)buf + 256;
    if (cudaMemset(buf, 0, 256) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    if (precision == TRSTMI_FP64) {
      if (cudaMemcpy((char*)buf + 256, phi, nd * sizeof(double2), cudaMemcpyHostToDevice) ||
          launch_gram_f64(N, d, 1, src, (unsigned long long*)buf, num_sms, 0)) {
        rc = TRSTMI_ECUDA; break;
      }
      unsigned long long b = 0;
      if (cudaMemcpy(&b, buf, sizeof(b), cudaMemcpyDeviceToHost)) { rc = TRSTMI_ECUDA; break; }
      std::memcpy(mu2, &b, sizeof(double));
    } else {
      f32.resize(2 * nd);
      for (size_t e = 0; e < 2 * nd; ++e) f32[e] = (float)phi[e];
      if (cudaMemcpy((char*)buf + 256, f32.data(), nd * sizeof(float2), cudaMemcpyHostToDevice) ||
          launch_gram_f32(N, d, 1, src, (unsigned int*)buf, nullptr, num_sms, 0)) {
        rc = TRSTMI_ECUDA; break;
      }
      unsigned int b = 0;
      if (cudaMemcpy(&b, buf, sizeof(b), cudaMemcpyDeviceToHost)) { rc = TRSTMI_ECUDA; break; }
      float f;
      std::memcpy(&f, &b, sizeof(f));
      *mu2 = (double)f;
    }
  } while (0);
  cudaFree(buf);
  return rc;
}

int trstmi_profile_score(trstmi_handle h, int precision, int launches, double delta,
                         size_t flush_bytes, double* avg_ms) {
  if (!h || launches < 1 || !avg_ms || !(delta >= 0)) return TRSTMI_EINVAL;
  if (precision < TRSTMI_FP64 || precision > TRSTMI_TF32_SCREEN) return TRSTMI_EINVAL;
  if (is_screen(precision) && !screen_supported(h->N, h->d, screen_fmt_of(precision, h->d)))
    return TRSTMI_EUNSUPPORTED;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  const int K = h->opt.K;
  void* flush = nullptr;
  if (flush_bytes) TRY_CUDA(h->dmem.allocate(&flush, flush_bytes));
  std::vector<cudaEvent_t> ev(2 * launches, nullptr);
  int rc = TRSTMI_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = TRSTMI_ECUDA;
  for (int l = 0; l < launches && rc == TRSTMI_OK; ++l) {
    if (flush && cudaMemsetAsync(flush, l & 0xff, flush_bytes, s) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    if (cudaMemsetAsync(h->mu2_k64, 0, (size_t)K * sizeof(unsigned long long), s) ||
        cudaMemsetAsync(h->mu2_k32, 0, (size_t)K * sizeof(unsigned int), s)) { rc = TRSTMI_ECUDA; break; }
    GramSource src{};
    src.perturb = true;
    src.seed = h->seed;
    src.t = (uint32_t)(l + 1);
    src.delta = delta;
    cudaEventRecord(ev[2 * l], s);
    cudaError_t e;
    if (precision == TRSTMI_FP64) {
      src.phi = h->phi64;
      e = launch_gram_f64(h->N, h->d, K, src, h->mu2_k64, h->num_sms, s);
    } else if (precision == TRSTMI_FP32) {
      // the scoring pass of the binary32 iteration: the candidates drawn once
      // (when the instance has room for them), then the tile pass
      src.phi = h->phi32;
      e = cudaSuccess;
      if (h->planes) {
        e = launch_gen_planes_f32(h->N, h->d, K, h->phi32, h->seed, 0u, nullptr, src.t, delta,
                                  h->planes, s);
        src.planes = h->planes;
      }
      if (e == cudaSuccess)
        e = launch_gram_f32(h->N, h->d, K, src, h->mu2_k32, nullptr, h->num_sms, s);
    } else {
      e = launch_screen(screen_fmt_of(precision, h->d), h->N, h->d, h->seed, h->phi32, K, 0u,
                        (uint32_t)(l + 1), delta, nullptr, h->mu2_k32, &h->misc[1], h->num_sms, s);
    }
    cudaEventRecord(ev[2 * l + 1], s);
    if (e != cudaSuccess) rc = record_cuda_error(e, "profiled kernel launch", __LINE__);
  }
  if (rc == TRSTMI_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = TRSTMI_ECUDA;
  double total = 0.0;
  if (rc == TRSTMI_OK) {
    for (int l = 0; l < launches; ++l) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * l], ev[2 * l + 1]) != cudaSuccess) rc = TRSTMI_ECUDA;
      total += ms;
    }
  }
  for (auto& e : ev) if (e) cudaEventDestroy(e);
  cudaStreamSynchronize(s);
  h->dmem.release(flush);
  if (rc == TRSTMI_OK) *avg_ms = total / launches;
  return rc;
}

namespace {
int lse_check(int N, int d, int count, double delta, int precision) {
  if (N < 2 || d < 1 || d > kMaxD || count < 1) return TRSTMI_EINVAL;
  if (!(delta > 0.0) || !(delta < INFINITY)) return TRSTMI_EINVAL;
  if (precision != TRSTMI_FP64 && precision != TRSTMI_FP32) return TRSTMI_EINVAL;
  if ((long long)count * N * d >= (1ll << 31)) return TRSTMI_ESIZE;
  return TRSTMI_OK;
}
}  // namespace

int trstmi_lse_scratch_bytes(int N, int d, int count, int precision, size_t* bytes) {
  if (!bytes) return TRSTMI_EINVAL;
  const int rc = lse_check(N, d, count, 1.0, precision);
  if (rc) return rc;
  *bytes = lse_scratch_bytes(N, d, count, precision == TRSTMI_FP64);
  return TRSTMI_OK;
}

int trstmi_lse_frames_device(int N, int d, int count, const double* v_dev, double delta,
                             int precision, void* scratch_dev, size_t scratch_bytes,
                             double* out_dev, double* grad_dev, void* stream) {
  trstmi::TraceRange trace_range("trstmi_lse_frames_device");
  int rc = lse_check(N, d, count, delta, precision);
  if (rc) return rc;
  if (!v_dev || !scratch_dev || !out_dev) return TRSTMI_EINVAL;
  if (scratch_bytes < lse_scratch_bytes(N, d, count, precision == TRSTMI_FP64))
    return TRSTMI_EINVAL;
  if (reinterpret_cast<uintptr_t>(scratch_dev) % 256 != 0) return TRSTMI_EINVAL;
  int dev = 0, num_sms = 0;
  if ((rc = caller_device(&dev)) != TRSTMI_OK) return rc;
  if ((rc = ensure_device(dev, &num_sms)) != TRSTMI_OK) return rc;
  TRY_CUDA(launch_lse(N, d, count, v_dev, delta, precision == TRSTMI_FP64, scratch_dev, out_dev,
                      grad_dev, num_sms, static_cast<cudaStream_t>(stream)));
  return TRSTMI_OK;
}

int trstmi_lse_frames(int N, int d, int count, const double* v, double delta, int precision,
                      double* F, double* s, double* grad) {
  trstmi::TraceRange trace_range("trstmi_lse_frames");
  int rc = lse_check(N, d, count, delta, precision);
  if (rc) return rc;
  if (!v || !F) return TRSTMI_EINVAL;
  int num_sms = 0, dev = 0;
  if ((rc = caller_device(&dev)) != TRSTMI_OK) return rc;
  if ((rc = ensure_device(dev, &num_sms)) != TRSTMI_OK) return rc;
  const size_t nv = (size_t)count * N * d * sizeof(double2);
  const size_t nscratch = lse_scratch_bytes(N, d, count, precision == TRSTMI_FP64);
  const size_t o_out = align_up(nv, 256), o_grad = align_up(o_out + 2 * sizeof(double) * count, 256);
  const size_t o_scr = align_up(o_grad + (grad ? nv : 0), 256);
  void* buf = nullptr;
  TRY_CUDA(cudaMalloc(&buf, o_scr + nscratch));
  char* b = static_cast<char*>(buf);
  std::vector<double> out(2 * (size_t)count);
  do {
    cudaError_t e = cudaMemcpy(b, v, nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = launch_lse(N, d, count, reinterpret_cast<const double*>(b), delta,
                     precision == TRSTMI_FP64, b + o_scr, reinterpret_cast<double*>(b + o_out),
                     grad ? reinterpret_cast<double*>(b + o_grad) : nullptr, num_sms, 0);
    if (e == cudaSuccess)
      e = cudaMemcpy(out.data(), b + o_out, out.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && grad) e = cudaMemcpy(grad, b + o_grad, nv, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { rc = record_cuda_error(e, "smooth maximum", __LINE__); break; }
    for (int q = 0; q < count; ++q) {
      if (std::isnan(out[2 * q])) { rc = TRSTMI_EINVAL; break; }   // a zero column
      F[q] = out[2 * q];
      if (s) s[q] = out[2 * q + 1];
    }
  } while (0);
  cudaFree(buf);
  return rc;
}

namespace {
int certificates_of(int N, int d, const double* v_dev, double tol, int num_sms,
                    cudaStream_t s, trstmi_certificates* out,
                    const DeviceMemory& dmem = DeviceMemory()) {
  void* scr = nullptr;
  TRY_CUDA(dmem.allocate(&scr, diag_scratch_bytes(N, d, tol)));
  unsigned char res[24];
  cudaError_t e = launch_diagnostics(N, d, v_dev, tol, scr, num_sms, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, scr, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) cudaStreamSynchronize(s);
  dmem.release(scr);
  if (e != cudaSuccess) return record_cuda_error(e, "certificates", __LINE__);
  uint32_t runs = 0, bad = 0;
  double mx = 0, mn = 0;
  std::memcpy(&mx, res, 8);
  std::memcpy(&mn, res + 8, 8);
  std::memcpy(&runs, res + 16, 4);
  std::memcpy(&bad, res + 20, 4);
  if (bad) return TRSTMI_EINVAL;
  trstmi_certificates c{};
  c.mu = std::sqrt(mx);
  c.mu_min = std::sqrt(mn);
  c.welch = N > d ? std::sqrt((double)(N - d) / ((double)d * (N - 1))) : 0.0;
  const bool above = d > 1 && (long long)N > (long long)d * d;
  c.orthoplex = above ? 1.0 / std::sqrt((double)d) : 0.0;
  c.levenshtein = above ? std::sqrt((2.0 * N - (double)d * (d + 1)) /
                                    (((double)N - d) * (d + 1.0))) : 0.0;
  c.lower_bound = std::max(c.welch, std::max(c.orthoplex, c.levenshtein));
  c.gap = c.mu - c.lower_bound;
  c.min_chordal = std::sqrt(std::max(0.0, 1.0 - mx));
  c.distinct = (int32_t)runs;
  *out = c;
  return TRSTMI_OK;
}
}  // namespace

int trstmi_frame_certificates(int N, int d, const double* phi, double tol,
                              trstmi_certificates* out) {
  trstmi::TraceRange trace_range("trstmi_frame_certificates");
  if (N < 2 || d < 1 || d > kMaxD || !phi || !out || !(tol >= 1e-7 && tol <= 1.0))
    return TRSTMI_EINVAL;
  int num_sms = 0, dev = 0;
  int rc = caller_device(&dev);
  if (rc || (rc = ensure_device(dev, &num_sms)) != TRSTMI_OK) return rc;
  const size_t nv = (size_t)N * d * sizeof(double2);
  void* v = nullptr;
  TRY_CUDA(cudaMalloc(&v, nv));
  cudaError_t e = cudaMemcpy(v, phi, nv, cudaMemcpyHostToDevice);
  rc = e == cudaSuccess ? certificates_of(N, d, static_cast<const double*>(v), tol, num_sms, 0, out)
                        : record_cuda_error(e, "certificates copy", __LINE__);
  cudaFree(v);
  return rc;
}

int trstmi_instance_certificates(trstmi_handle h, double tol, trstmi_certificates* out) {
  trstmi::TraceRange trace_range("trstmi_instance_certificates");
  if (!h || !out || !(tol >= 1e-7 && tol <= 1.0)) return TRSTMI_EINVAL;
  USE_DEVICE(h->opt.device);
  return certificates_of(h->N, h->d, reinterpret_cast<const double*>(h->phi64), tol,
                         h->num_sms, h->stream, out, h->dmem);
}

void trstmi_tr_default_options(trstmi_tr_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  const double ds[] = {0.1, 0.03, 0.01, 0.003, 0.001, 3e-4, 1e-4};
  o->n_delta = 7;
  for (int k = 0; k < 7; ++k) o->delta[k] = ds[k];
  o->max_outer = 100;
  o->max_cg = 200;
  o->radius0 = 0.1;
  o->radius_max = 1.0;
  o->eta = 1e-4;
  o->gtol = 1e-9;
  o->fd_step = 1e-6;
}

namespace {
int tr_check(int N, int d, const trstmi_tr_options* o) {
  if (N < 2 || d < 1 || d > kMaxD || !o) return TRSTMI_EINVAL;
  if (o->n_delta < 1 || o->n_delta > 16 || o->max_outer < 0 || o->max_cg < 1) return TRSTMI_EINVAL;
  if (o->path < 0 || o->path > 2) return TRSTMI_EINVAL;
  for (int k = 0; k < o->n_delta; ++k)
    if (!(o->delta[k] > 0.0) || !(o->delta[k] < INFINITY)) return TRSTMI_EINVAL;
  if (!(o->radius0 > 0.0) || !(o->radius_max >= o->radius0) || !(o->eta >= 0.0 && o->eta < 0.25) ||
      !(o->gtol >= 0.0) || !(o->fd_step > 0.0) || (o->hessian != 0 && o->hessian != 1))
    return TRSTMI_EINVAL;
  if ((long long)N * d >= (1ll << 28)) return TRSTMI_ESIZE;
  return TRSTMI_OK;
}
}  // namespace

namespace {
int tr_solve_on(int device, int N, int d, double* phi, const trstmi_tr_options* o,
                trstmi_tr_row* trace, int cap, int* n_rows,
                const DeviceMemory& dmem = DeviceMemory()) {
  int rc = tr_check(N, d, o);
  if (rc) return rc;
  if (!phi || cap < 0) return TRSTMI_EINVAL;
  int num_sms = 0;
  USE_DEVICE(device);
  if ((rc = ensure_device(device, &num_sms)) != TRSTMI_OK) return rc;
  const size_t nv = (size_t)N * d * sizeof(double2);
  const size_t o_scr = align_up(nv, 256);
  void* buf = nullptr;
  TRY_CUDA(dmem.allocate(&buf, o_scr + tr_device_bytes(N, d, 1, cap, o->hessian)));
  char* b = static_cast<char*>(buf);
  cudaError_t e = cudaMemcpy(b, phi, nv, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    TrFrameLog log{trace, cap, 0, 0.0, 0};
    rc = tr_solve_device(N, d, 1, reinterpret_cast<double*>(b), *o, b + o_scr, num_sms, 0, &log);
    if (n_rows) *n_rows = log.n;
    if (rc == TRSTMI_OK && cudaMemcpy(phi, b, nv, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = TRSTMI_ECUDA;
  } else {
    rc = record_cuda_error(e, "trust-region frame copy", __LINE__);
  }
  cudaStreamSynchronize(0);
  dmem.release(buf);
  return rc;
}
}  // namespace

int trstmi_tr_solve(int N, int d, double* phi, const trstmi_tr_options* o, trstmi_tr_row* trace,
                    int cap, int* n_rows) {
  trstmi::TraceRange trace_range("trstmi_tr_solve");
  int dev = 0;
  const int rc = caller_device(&dev);
  return rc ? rc : tr_solve_on(dev, N, d, phi, o, trace, cap, n_rows);
}

int trstmi_tr_multistart(int N, int d, uint64_t seed0, int L, const trstmi_tr_options* o,
                         int batch_cap, trstmi_multistart_result* out, double* mu_all,
                         double* best_phi, trstmi_tr_row* trace, int cap, int* n_rows,
                         int* work) {
  trstmi::TraceRange trace_range("trstmi_tr_multistart");
  int rc = tr_check(N, d, o);
  if (rc) return rc;
  if (!out || cap < 0) return TRSTMI_EINVAL;
  if (L <= 0) L = 2 * d * d;
  const int B = batch_cap > 0 ? std::min(batch_cap, L) : L;
  int num_sms = 0, dev = 0;
  if ((rc = caller_device(&dev)) != TRSTMI_OK) return rc;
  if ((rc = ensure_device(dev, &num_sms)) != TRSTMI_OK) return rc;
  const size_t nv = (size_t)N * d * sizeof(double2);
  const size_t o_f32 = align_up(nv * B, 256);
  const size_t o_scr = o_f32 + align_up(nv / 2, 256);
  void* buf = nullptr;
  TRY_CUDA(cudaMalloc(&buf, o_scr + tr_device_bytes(N, d, B, 0, o->hessian)));
  char* b = static_cast<char*>(buf);
  std::vector<double> mu(L);
  std::vector<TrFrameLog> logs(B);
  int best = 0;
  for (int b0 = 0; b0 < L && rc == TRSTMI_OK; b0 += B) {
    const int n = std::min(B, L - b0);
    // every trial starts from the frame trstmi_create draws for its seed
    for (int i = 0; i < n; ++i) {
      cudaError_t e = launch_init_frame(N, d, seed0 + (uint64_t)(b0 + i),
                                        reinterpret_cast<double2*>(b + nv * i),
                                        reinterpret_cast<float2*>(b + o_f32), nullptr, 0);
      if (e != cudaSuccess) { rc = record_cuda_error(e, "trial initialisation", __LINE__); break; }
    }
    if (rc) break;
    for (int i = 0; i < n; ++i) logs[i] = TrFrameLog{nullptr, 0, 0, 0.0, 0};
    rc = tr_solve_device(N, d, n, reinterpret_cast<double*>(b), *o, b + o_scr, num_sms, 0,
                         logs.data());
    if (rc) break;
    for (int i = 0; i < n; ++i) {
      if (work) {
        work[2 * (size_t)(b0 + i)] = logs[i].n;
        work[2 * (size_t)(b0 + i) + 1] = logs[i].hv_products;
      }
      mu[b0 + i] = std::sqrt(logs[i].mu2);
      if (b0 + i == 0 || mu[b0 + i] < mu[best]) {
        best = b0 + i;
        if (best_phi && cudaMemcpy(best_phi, b + nv * i, nv, cudaMemcpyDeviceToHost) != cudaSuccess)
          rc = TRSTMI_ECUDA;
      }
    }
  }
  cudaFree(buf);
  if (rc) return rc;
  out->mu = mu[best];
  out->best = best;
  out->trials = L;
  out->best_seed = seed0 + (uint64_t)best;
  if (mu_all) std::copy(mu.begin(), mu.end(), mu_all);
  if (n_rows) *n_rows = 0;
  if (trace || n_rows) {
    // the winning trial alone again: the same trajectory, so the same rows
    void* one = nullptr;
    TRY_CUDA(cudaMalloc(&one, align_up(nv, 256) + align_up(nv / 2, 256) + tr_device_bytes(N, d, 1, cap, o->hessian)));
    char* c = static_cast<char*>(one);
    cudaError_t e = launch_init_frame(N, d, out->best_seed, reinterpret_cast<double2*>(c),
                                      reinterpret_cast<float2*>(c + align_up(nv, 256)), nullptr, 0);
    TrFrameLog log{trace, cap, 0, 0.0, 0};
    if (e == cudaSuccess)
      rc = tr_solve_device(N, d, 1, reinterpret_cast<double*>(c), *o,
                           c + align_up(nv, 256) + align_up(nv / 2, 256), num_sms, 0, &log);
    else
      rc = record_cuda_error(e, "trial initialisation", __LINE__);
    if (n_rows) *n_rows = log.n;
    cudaFree(one);
  }
  return rc;
}

int trstmi_instance_tr_solve(trstmi_handle h, const trstmi_tr_options* o, trstmi_tr_row* trace,
                             int cap, int* n_rows) {
  if (!h) return TRSTMI_EINVAL;
  std::vector<double> phi(2 * (size_t)h->N * h->d);
  int rc = trstmi_get_phi(h, phi.data());
  if (rc) return rc;
  if ((rc = tr_solve_on(h->opt.device, h->N, h->d, phi.data(), o, trace, cap, n_rows,
                        h->dmem)) !=
      TRSTMI_OK)
    return rc;
  return trstmi_set_phi(h, phi.data());
}

int trstmi_screen_wait_test(trstmi_handle h, int precision, double wait_limit_ms) {
  if (!h || !is_screen_precision(precision)) return TRSTMI_EINVAL;
  if (!(wait_limit_ms > 0.0 && wait_limit_ms <= 2000.0)) return TRSTMI_EINVAL;
  if (!screen_supported(h->N, h->d, screen_fmt_of(precision, h->d))) return TRSTMI_EUNSUPPORTED;
  USE_DEVICE(h->opt.device);
  cudaStream_t s = h->stream;
  const int count = std::min(h->opt.K, 8);
  TRY_CUDA(cudaMemsetAsync(&h->misc[1], 0, sizeof(uint32_t), s));
  TRY_CUDA(launch_screen_wait_test(screen_fmt_of(precision, h->d), h->N, h->d, h->phi32, count,
                                   h->mu2_k32, &h->misc[1],
                                   (unsigned long long)(wait_limit_ms * 1e6), h->num_sms, s));
  uint32_t err = 0;
  TRY_CUDA(cudaMemcpyAsync(&err, &h->misc[1], sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TRY_CUDA(cudaStreamSynchronize(s));
  return (err & kErrTimeout) ? TRSTMI_ETIMEOUT : TRSTMI_OK;
}

}  // extern "C"
