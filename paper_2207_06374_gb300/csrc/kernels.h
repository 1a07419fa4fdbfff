// Host-side launchers of the TRSTMI kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>
#include "common.cuh"
#include "../../include/trstmi.h"

namespace trstmi {

// Makes a device current for the guard's lifetime and restores the calling
// thread's current device when the guard goes out of scope, so an entry
// point never leaves its caller bound to another GPU.
class DeviceGuard {
 public:
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev_) != cudaSuccess) { cudaGetLastError(); prev_ = -1; }
    if (prev_ == device) { ok_ = true; return; }
    ok_ = cudaSetDevice(device) == cudaSuccess;
    if (!ok_) cudaGetLastError();
    restore_ = ok_ && prev_ >= 0;
  }
  ~DeviceGuard() {
    if (restore_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;

 private:
  int prev_ = -1;
  bool ok_ = false, restore_ = false;
};

// Device memory of one handle: the caller's allocator when its options carry
// one (trstmi_options::dev_alloc / dev_free), cudaMalloc / cudaFree otherwise.
struct DeviceMemory {
  void* (*alloc_fn)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* ctx = nullptr;
  DeviceMemory() = default;
  explicit DeviceMemory(const trstmi_options& o)
      : alloc_fn(o.dev_alloc), free_fn(o.dev_free), ctx(o.alloc_ctx) {}
  // both callbacks or neither
  static bool valid(const trstmi_options& o) { return (o.dev_alloc == nullptr) == (o.dev_free == nullptr); }
  // cudaErrorMemoryAllocation when the callback returns NULL or memory that
  // is not 256-byte aligned (that memory is handed back)
  cudaError_t allocate(void** p, size_t bytes) const {
    if (!alloc_fn) return cudaMalloc(p, bytes);
    *p = alloc_fn(bytes, ctx);
    if (*p && reinterpret_cast<uintptr_t>(*p) % 256 != 0) {
      free_fn(*p, ctx);
      *p = nullptr;
    }
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  void release(void* p) const {
    if (!p) return;
    if (alloc_fn) free_fn(p, ctx); else cudaFree(p);
  }
};

// Operand format of the tensor-core screen: bf16 / fp16 / tf32 for d <= 32,
// and the wide bf16 / fp16 layouts (two 128-byte atoms per column) for
// 32 < d <= 64.
enum ScreenFmt : int {
  kScreenBF16 = 0, kScreenFP16 = 1, kScreenTF32 = 2, kScreenBF16W = 3, kScreenFP16W = 4
};
inline bool is_screen_precision(int p) {
  return p == TRSTMI_BF16_SCREEN || p == TRSTMI_FP16_SCREEN || p == TRSTMI_TF32_SCREEN;
}
inline int screen_fmt_of(int precision, int d) {
  if (precision == TRSTMI_TF32_SCREEN) return kScreenTF32;
  const bool wide = d > 32;
  return precision == TRSTMI_FP16_SCREEN ? (wide ? kScreenFP16W : kScreenFP16)
                                         : (wide ? kScreenBF16W : kScreenBF16);
}

// Which frame a Gram pass reads.
struct GramSource {
  // perturb = true: candidate c of iteration t around phi (binary32 or
  // binary64 per the pass's precision), c = cand_list[slot] or c0 + slot.
  // perturb = false: frame(s) read from phi + slot*d*N, optionally
  // renormalised on load.
  bool perturb;
  const void* phi;              // float2* or double2*
  uint64_t seed;
  const uint32_t* cand_list;    // nullable
  uint32_t c0;
  uint32_t t;                   // used when st == nullptr
  double delta;                 // used when st == nullptr
  const DevState* st;           // nullable: t = st->t + 1, delta = st->delta_used, skip unless active
  bool normalize;               // frame source only
  const uint32_t* gate;         // nullable: skip the pass unless *gate != 0
  // perturb with planes != nullptr: slot s's candidate was drawn already (by
  // launch_gen_planes) into planes + s * 2dN as [i][column] planes of real then
  // imaginary parts; the pass reads it instead of drawing it per tile
  const void* planes;
};

// Draws candidates c0 .. c0+count-1 (with st: of the next iteration, t + 1
// and the radius in use, nothing unless st->active, zero columns set
// kErrZeroColumn; without: of iteration t with radius delta) around the
// binary32 frame into [i][column] planes, slot s at planes + s * 2dN floats.
// One thread per column, the arithmetic of the tile pass.
cudaError_t launch_gen_planes_f32(int N, int d, int count, const float2* phi, uint64_t seed,
                                  uint32_t c0, DevState* st, uint32_t t, double delta,
                                  float* planes, cudaStream_t s,
                                  const uint32_t* cand_list = nullptr,
                                  const uint32_t* gate = nullptr);

// Optional pair filter of the binary32 certification pass.
struct PairFilter {
  const unsigned int* mu2_ref;  // binary32 max |G|^2 of the same frame (bits)
  float margin;                 // on |G|: keep pairs with |G| >= sqrt(ref) - margin
  uint2* pairs;
  uint32_t* npairs;
  uint32_t cap;
  uint32_t* overflow;
  // nullable: binary64 bits of a factor the margin is multiplied by (the
  // largest squared column norm of a frame whose columns are not unit)
  const unsigned long long* scale_bits;
  // mu2_ref is a hint within this much (on mu^2) of the frame's binary32 max
  // rather than that max itself (0: it is the max)
  float ref_slack_mu2;
  // nonzero: no reference is read; each tile keeps its pairs within the
  // margin of the tile's own maximum (at most the frame's, so the kept set
  // holds every pair within the margin of the frame's maximum), and the max
  // and the pair list come from one pass
  int local;
};

// Lower end of the kept range of |G|: sqrt(binary32 max, less the hint's
// slack) - margin (scaled).
__device__ __forceinline__ float filter_lo(const PairFilter& f) {
  const float ref = sqrtf(fmaxf(__uint_as_float(*f.mu2_ref) - f.ref_slack_mu2, 0.0f));
  float margin = f.margin;
  if (f.scale_bits) margin = (float)((double)margin * __longlong_as_double((long long)*f.scale_bits));
  return fmaxf(ref - margin, 0.0f);
}

// mu^2 per slot: max over j<k of |G_jk|^2, atomically maxed into out[slot]
// (unsigned int bits for binary32, unsigned long long bits for binary64).
cudaError_t launch_gram_f32(int N, int d, int nslots, const GramSource& src,
                            unsigned int* out, const PairFilter* filter, int num_sms,
                            cudaStream_t s);
cudaError_t launch_gram_f64(int N, int d, int nslots, const GramSource& src,
                            unsigned long long* out, int num_sms, cudaStream_t s);

// Largest d the Gram kernels support.
constexpr int kMaxD = 256;

cudaError_t launch_init_frame(int N, int d, uint64_t seed, double2* phi64, float2* phi32,
                              DevState* st, cudaStream_t s);
// call_iters (nonzero): this is the first iteration of a trstmi_step call of
// that many iterations, and the kernel also sets the call's stop and start
// counters (k_set_stop's work)
cudaError_t launch_iter_begin(DevState* st, void* zero0, size_t bytes0, void* zero1,
                              size_t bytes1, void* zero2, size_t bytes2, cudaStream_t s,
                              uint32_t call_iters = 0);
// plain modes: argmin over K candidates, accept/radius rule, trace row
cudaError_t launch_select_decide_f32(DevState* st, const unsigned int* mu2, int K,
                                     TraceRowDev* trace, cudaStream_t s);
cudaError_t launch_select_decide_f64(DevState* st, const unsigned long long* mu2, int K,
                                     TraceRowDev* trace, cudaStream_t s);
// plain modes: regenerate the accepted candidate in place
cudaError_t launch_commit_f32(int N, int d, uint64_t seed, DevState* st, float2* phi32,
                              double2* phi64, cudaStream_t s);
cudaError_t launch_commit_f64(int N, int d, uint64_t seed, DevState* st, double2* phi64,
                              float2* phi32, cudaStream_t s);
// screen mode
cudaError_t launch_topk(DevState* st, const unsigned int* mu2_screen, int K, int k,
                        uint32_t* topk, unsigned int* mu2_top, cudaStream_t s);
// hint_out (nullable): receives the chosen survivor's binary32 score bits
// when it is certified (the certification's filter hint).
// sel (nullable): sel[0] receives the winner's survivor slot and sel[1] 1 when
// its certification needs the binary32 filter pass (its pair list from the
// survivor pair pass, list_count / list_cap, is missing or overflowed); with
// filter_available false such a winner sets st->overflow instead (the full
// binary64 pass).
cudaError_t launch_materialize64(int N, int d, uint64_t seed, DevState* st,
                                 const uint32_t* topk, const unsigned int* mu2_top, int k,
                                 const double2* phi64, double2* cand64, float2* cand32,
                                 cudaStream_t s, unsigned int* hint_out = nullptr,
                                 const uint32_t* list_count = nullptr, uint32_t list_cap = 0,
                                 uint32_t* sel = nullptr, bool filter_available = true);
// hint_bits / own_bits (nullable): the filter pass ran from a hint (its
// slack hint_slack_mu2) instead of the frame's binary32 max; if the hint less
// its slack exceeds the pass's own max (own_bits), the kept set may miss the
// maximum pair and *overflow is set, so the full binary64 pass runs.
cudaError_t launch_pairs64(const uint32_t* active, const uint32_t* npairs, const uint2* pairs,
                           uint32_t cap, int d, const double2* frame64, unsigned long long* out,
                           cudaStream_t s, const unsigned int* hint_bits = nullptr,
                           const unsigned int* own_bits = nullptr, float hint_slack_mu2 = 0.f,
                           uint32_t* overflow = nullptr, const uint32_t* sel = nullptr,
                           const uint2* lists = nullptr, const uint32_t* list_count = nullptr,
                           uint32_t list_cap = 0);
// Binary64 mu^2 of a normalised frame into *cert64 by the certification
// passes (binary32 max into cert32[0], filter pass into cert32[1] / pairs /
// *npairs, binary64 over the kept pairs, all pairs when *overflow is set);
// cert32[0..1], *cert64, *npairs and *overflow zero before.  active: gate.
cudaError_t launch_frame_certify(int N, int d, const double2* p64, const float2* p32,
                                 unsigned int* cert32, unsigned long long* cert64, uint2* pairs,
                                 uint32_t cap, uint32_t* npairs, uint32_t* overflow,
                                 const uint32_t* active, int num_sms, cudaStream_t s);
// |G| margin between a frame's binary32 and binary64 Gram entries
float certify_margin(int d);
// sel (nullable, from launch_materialize64): when sel[1] is 0 the pairs are the
// winner's list, lists + sel[0] * list_cap (list_count[sel[0]] of them),
// instead of pairs / npairs, and the hint check is skipped.
// binary32 |G|^2 of each survivor's listed pairs (lists, k x cap; count[s]
// above cap: left to the full pass), the pair's two columns of candidate
// topk[s] drawn by one warp with the bits of the survivors' binary32 draw,
// maxed into mu2[s] with the bits the binary32 tile pass gives those pairs.
// Returns at once unless the iteration in st is active and screened; d <= 64.
cudaError_t launch_pairs32(DevState* st, const uint2* lists, const uint32_t* count,
                           uint32_t cap, int k, int N, int d, const float2* phi, uint64_t seed,
                           const uint32_t* topk, unsigned int* mu2, cudaStream_t s);
// The accept/radius rule on the certified binary64 mu^2 (or, uncertified, on
// the survivor's binary32 score) with its trace row, and the copy of the
// accepted candidate into the frame, in one launch; *done is a
// zero-initialised counter the launch leaves at zero
cudaError_t launch_decide_commit(int N, int d, DevState* st, const unsigned long long* mu2_64,
                                 TraceRowDev* trace, const double2* cand64, const float2* cand32,
                                 double2* phi64, float2* phi32, unsigned int* done,
                                 cudaStream_t s);
// frame utilities
cudaError_t launch_normalize64(int N, int d, const double2* in, double2* out64, float2* out32,
                               DevState* st, cudaStream_t s);
cudaError_t launch_gen_candidate(int N, int d, uint64_t seed, uint32_t t, uint32_t c,
                                 double delta, bool f64, const double2* phi64,
                                 const float2* phi32, double2* out, cudaStream_t s);

// tensor-core screen (tc_screen.cu)
// d <= 32 (bf16, fp16, tf32) or d <= 64 (wide bf16, fp16), 2 <= N <= 65536
bool screen_supported(int N, int d, int fmt);
// One instance as the batched screen sees it (device table).
struct ScreenSlot {
  const float2* phi32;
  unsigned int* mu2;     // K screen scores
  const DevState* st;
  uint64_t seed;
  int N, d;
};
// Screen of (instance, candidate) items of many instances; an instance's items
// are skipped unless it is active and ranks with the screen this iteration.
cudaError_t launch_screen_batched(int fmt, const ScreenSlot* slots, const uint2* items,
                                  int n_items, uint32_t* err_flag, int num_sms, cudaStream_t s);

// fmt: ScreenFmt of the operands.  With st, runs only when st->active &&
// st->use_screen.
cudaError_t launch_screen(int fmt, int N, int d, uint64_t seed, const float2* phi32, int K,
                          uint32_t c0, uint32_t t, double delta, const DevState* st,
                          unsigned int* mu2_out, uint32_t* err_flag, int num_sms,
                          cudaStream_t s);

// The screen over K candidates with its block producers withheld: no column
// block is ever filled, so the MMA issuer's first wait runs out after
// wait_limit_ns (at most the default bound), sets err_flag's timeout bit and
// every role of each CTA leaves.  Exercises the bounded waits.
// Survivor pair pass (tc_screen.cu): for each of the k survivors (candidate
// topk[s] of the iteration in st, screen score mu2[topk[s]]), the pairs whose
// screened |G| is at least sqrt(score) - 2 err go to pairs[s * cap ..] with
// count[s] (zeroed before); count[s] > cap marks an overflowed list and sets
// *overflow_any.  Returns at once unless the iteration is active and screened.
cudaError_t launch_screen_pairs(int fmt, int N, int d, uint64_t seed, const float2* phi32,
                                const DevState* st, const uint32_t* topk,
                                const unsigned int* mu2, int k, float err, uint2* pairs,
                                uint32_t* count, uint32_t cap, uint32_t* overflow_any,
                                uint32_t* err_flag, int num_sms, cudaStream_t s,
                                unsigned char* blocks = nullptr);
// blocks (nullable): room for the k survivors' column blocks (k x nb x
// screen_block_bytes(fmt)), drawn once by a first launch and copied by the
// pair pass instead of each item drawing its two blocks.
// the err of launch_screen_pairs for screen format fmt
float screen_pair_err(int fmt);
// bytes of one 128-column block in screen format fmt
size_t screen_block_bytes(int fmt);
cudaError_t launch_screen_wait_test(int fmt, int N, int d, const float2* phi32, int K,
                                    unsigned int* mu2_out, uint32_t* err_flag,
                                    unsigned long long wait_limit_ns, int num_sms,
                                    cudaStream_t s);

// ------------------------------------------ trust-region procedure (tr.cu)
// L frames advance together, each exactly as it would alone.  Device bytes
// the procedure needs beside the frames; v_dev (L x N x d complex doubles)
// is replaced by the results.  logs (nullable, L entries): each frame's trace
// rows (up to cap; n counts them all), its final max |G_jk|^2 and Hessian
// products.  Returns a TRSTMI_ status.
struct TrFrameLog {
  trstmi_tr_row* rows;
  int cap, n;
  double mu2;
  int hv_products;
};
size_t tr_device_bytes(int N, int d, int L, int trace_cap, int hessian);
int tr_solve_device(int N, int d, int L, double* v_dev, const trstmi_tr_options& o,
                    void* scratch, int num_sms, cudaStream_t s, TrFrameLog* logs);

// ------------------------------------------ certificates (diag.cu)
// max / min of |G_jk|^2 and the distinct distances at resolution tol of a
// frame (v: device, N x d complex interleaved doubles, normalised inside).
// Results at the start of scratch: [max bits u64][min bits u64][runs u32]
// [zero column u32].
size_t diag_scratch_bytes(int N, int d, double tol);
cudaError_t launch_diagnostics(int N, int d, const double* v_dev, double tol, void* scratch,
                               int num_sms, cudaStream_t s);
cudaError_t init_diag_attributes(int optin);

// ------------------------------------------ smooth maximum (lse.cu)
// F_{s,delta}, s and the gradient in V of `count` frames (v: device, count x
// N x d complex interleaved doubles); out: device, count x [F, s]; grad:
// device, count x N x d complex, or null.  Arithmetic in binary64 (f64) or
// binary32 (the sums of the tiles' weights, S, F and the final projection in
// binary64).
size_t lse_scratch_bytes(int N, int d, int count, bool f64);
cudaError_t launch_lse(int N, int d, int count, const double* v, double delta, bool f64,
                       void* scratch, double* out, double* grad, int num_sms, cudaStream_t s);
// The same with a smoothing parameter per frame (deltas: device, count doubles, > 0).
cudaError_t launch_lse_deltas(int N, int d, int count, const double* v, const double* deltas,
                              bool f64, void* scratch, double* out, double* grad, int num_sms,
                              cudaStream_t s);
cudaError_t init_lse_attributes(int optin);

// ------------------------------------------------------ batched searches
// One instance of a batch, as the batched kernels see it (device table).
struct SlotDesc {
  DevState* st;
  void* phi;            // frame in the scoring precision (float2* or double2*)
  void* phi_other;      // the other precision's copy (kept in step on commit)
  void* mu2;            // K candidate scores (u32 / u64 bit patterns)
  TraceRowDev* trace;
  uint64_t seed;
  int N, d, K;
  int R;                // tile width 16R of this instance's Gram pass (kResident: whole
                        // candidate in shared memory)
  int ntiles;           // upper-triangle tiles at that width
  int screen;           // screen modes: 1 if the tensor-core screen handles this shape
  // screen modes only: top-k survivors, their fp32 scores, the binary64
  // winner and its binary32 rounding, certification scratch
  uint32_t* topk;
  unsigned int* mu2_top;
  int topk_n;
  uint32_t pair_cap;
  double2* cand64;
  float2* cand32;
  unsigned int* cert32;          // [0] fp32 max of the winner, [1] filter pass's own max
  unsigned long long* cert64;    // certified binary64 mu^2 of the winner
  uint2* pairs;                  // preselected pairs (pair_cap)
};

// Passes of the batched scoring kernel.
enum BatchPassMode : int {
  kPassFull = 0,      // every candidate, binary32/64 (ranking when not screened)
  kPassRescore = 1,   // the top-k survivors, binary32, into mu2_top
  kPassFrameMax = 2,  // the winner's binary32 rounding: max |G|^2 into cert32[0] (the
                      // iteration uses the winner's score as that value's hint instead)
  kPassFilter = 3,    // same frame: pairs within the bound of cert32[0] into pairs
  kPassFrame64 = 4,   // the binary64 winner, all pairs, only after a pair-list overflow
};

// Iteration start for every instance (one CTA each); also zeroes the work
// counters.  screen_mode: instances with SlotDesc::screen rank with the
// tensor-core screen while their radius is >= screen_min_delta.
cudaError_t launch_batch_begin(SlotDesc* slots, int n, unsigned long long* counters, int ncounters,
                               bool f64, bool screen_mode, cudaStream_t s);
// Persistent scoring pass over the instances of one tile-width group: work
// items (instance, candidate-or-frame, tile) handed out by an atomic counter.
cudaError_t launch_batch_score(bool f64, int R, const SlotDesc* slots, const int* group,
                               const long long* group_begin, int ngroup, long long nitems,
                               unsigned long long* counter, size_t smem, int grid,
                               cudaStream_t s, int mode = kPassFull);
// Screen modes, one CTA (or column warps) per instance.
cudaError_t launch_batch_topk(SlotDesc* slots, int n, cudaStream_t s);
cudaError_t launch_batch_materialize64(SlotDesc* slots, int n, int maxN, cudaStream_t s);
cudaError_t launch_batch_pairs64(SlotDesc* slots, int n, cudaStream_t s);
cudaError_t launch_batch_decide_certified(SlotDesc* slots, int n, cudaStream_t s);
cudaError_t launch_batch_commit_copy(SlotDesc* slots, int n, int maxN, int maxd, cudaStream_t s);
cudaError_t launch_batch_decide(SlotDesc* slots, int n, bool f64, cudaStream_t s);
cudaError_t launch_batch_commit(SlotDesc* slots, int n, int maxN, bool f64, cudaStream_t s);
cudaError_t batch_score_occupancy(bool f64, int R, size_t smem, int* blocks_per_sm);
size_t gram_smem_bytes(bool f64, int d, int R);
// Whole-candidate scoring of small instances (SlotDesc::R == kResident):
// one CTA per (instance, candidate), the candidate drawn once into shared
// memory; modes kPassFull and kPassRescore.
constexpr int kResident = 0;
cudaError_t launch_batch_resident(bool f64, const SlotDesc* slots, const int* group,
                                  const long long* group_begin, int ngroup, long long nitems,
                                  unsigned long long* counter, size_t smem, int grid,
                                  cudaStream_t s, int mode);
cudaError_t batch_resident_occupancy(bool f64, size_t smem, int* blocks_per_sm);
size_t resident_smem_bytes(bool f64, int d, int N);
// Autotuned tile-width cache per (d, ceil log2 N): -1 if not measured yet,
// else R in {kResident, 1, 2, 4}.
int cached_width(bool f64, int d, int N);
void store_width(bool f64, int d, int N, int R);
int tiles_at_width(int N, int R);
bool width_feasible(bool f64, int d, int N, int R);

// Launch plan of one iteration over many instances (plan.cu): width-group
// tables of every scoring pass and the screen's work items, in device buffers
// allocated once for a capacity and refilled by rebuild().
struct BatchPlan {
  static constexpr int kPasses = 5;
  static constexpr int kCounters = 24;
  struct Group {
    int R = 1;
    bool f64 = false;
    int* d_ids = nullptr;
    long long* d_begin = nullptr;
    int count = 0;
    long long nitems = 0;
    size_t smem = 0;
    int grid = 0;
    int counter = 0;
  };
  struct Table { int* d_ids = nullptr; long long* d_begin = nullptr; };
  void* mem = nullptr;
  int cap_slots = 0;
  long long cap_items = 0;
  int num_sms = 0;
  int precision = 0;
  int maxN = 0, maxd = 0;
  int ncounters = 0;
  Table tables[kPasses][4];
  std::vector<Group> groups[kPasses];
  ScreenSlot* d_screen_slots = nullptr;
  uint2* d_items = nullptr;
  int n_items = 0;        // screen items; the last n_wide of them take the wide format
  int n_wide = 0;
  unsigned long long* d_counters = nullptr;
  // Large binary32 instances (N >= kPlanesMinN, scored in tiles): their
  // candidate passes draw each candidate once into the planes scratch and run
  // the double-buffered tile pass over them (the single-instance kernels, the
  // same bits as the shared pass), one instance after the other.
  static constexpr int kPlanesMinN = 384;
  void* planes = nullptr;
  size_t planes_bytes = 0;
  std::vector<SlotDesc> large;
  DeviceMemory dmem;      // where mem and planes come from (set before init)

  // planes_bytes: the scratch for large instances (0: none)
  int init(int capacity_slots, long long capacity_items, int num_sms, size_t planes_bytes = 0);
  void destroy();
  // h: host copy of the device slot table (R of every slot chosen)
  int rebuild(const std::vector<SlotDesc>& h, int precision, cudaStream_t s);
  int enqueue_iteration(SlotDesc* d_slots, int n, uint32_t* err, cudaStream_t s) const;
  // the screen of every item: one launch per operand format present
  cudaError_t launch_screen(uint32_t* err, cudaStream_t s) const;
  // a candidate pass (kPassFull or kPassRescore) of the large instances
  cudaError_t launch_large(int pass, cudaStream_t s) const;
  cudaError_t launch_pass(int pass, SlotDesc* d_slots, cudaStream_t s) const;
  int kernels_per_iteration() const;
};

cudaError_t init_kernel_attributes();
cudaError_t init_screen_attributes(int optin_smem);

}  // namespace trstmi
