// Host-side launchers of the TRSTMI kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "common.cuh"

namespace trstmi {

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
};

// Optional pair filter of the binary32 certification pass.
struct PairFilter {
  const unsigned int* mu2_ref;  // binary32 max |G|^2 of the same frame (bits)
  float margin;                 // on |G|: keep pairs with |G| >= sqrt(ref) - margin
  uint2* pairs;
  uint32_t* npairs;
  uint32_t cap;
  uint32_t* overflow;
};

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
cudaError_t launch_iter_begin(DevState* st, void* zero0, size_t bytes0, void* zero1,
                              size_t bytes1, void* zero2, size_t bytes2, cudaStream_t s);
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
                        uint32_t* topk, cudaStream_t s);
cudaError_t launch_materialize64(int N, int d, uint64_t seed, DevState* st,
                                 const uint32_t* topk, const unsigned int* mu2_top, int k,
                                 const double2* phi64, double2* cand64, float2* cand32,
                                 cudaStream_t s);
cudaError_t launch_pairs64(const uint32_t* active, const uint32_t* npairs, const uint2* pairs,
                           uint32_t cap, int d, const double2* frame64, unsigned long long* out,
                           cudaStream_t s);
cudaError_t launch_decide_certified(DevState* st, const unsigned long long* mu2_64,
                                    TraceRowDev* trace, cudaStream_t s);
cudaError_t launch_commit_copy(int N, int d, DevState* st, const double2* cand64,
                               const float2* cand32, double2* phi64, float2* phi32,
                               cudaStream_t s);
// frame utilities
cudaError_t launch_normalize64(int N, int d, const double2* in, double2* out64, float2* out32,
                               DevState* st, cudaStream_t s);
cudaError_t launch_gen_candidate(int N, int d, uint64_t seed, uint32_t t, uint32_t c,
                                 double delta, bool f64, const double2* phi64,
                                 const float2* phi32, double2* out, cudaStream_t s);

// tensor-core screen (tc_screen.cu)
bool screen_supported(int N, int d);
// fp16 = false: bf16 operands; true: fp16 operands.  With st, runs only when
// st->active && st->use_screen.
cudaError_t launch_screen(bool fp16, int N, int d, uint64_t seed, const float2* phi32, int K,
                          uint32_t c0, uint32_t t, double delta, const DevState* st,
                          unsigned int* mu2_out, uint32_t* err_flag, int num_sms,
                          cudaStream_t s);

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
  int R;                // tile width 16R of this instance's Gram pass
  int ntiles;           // upper-triangle tiles at that width
  int pad;
  long long item_begin; // first work item of this instance within its width group
};

// Iteration start for every instance (one CTA each); also zeroes the work counters.
cudaError_t launch_batch_begin(SlotDesc* slots, int n, unsigned long long* counters, int ncounters,
                               bool f64, cudaStream_t s);
// Persistent scoring pass over the instances of one tile-width group: work
// items (instance, candidate, tile) handed out by an atomic counter.
cudaError_t launch_batch_score(bool f64, int R, const SlotDesc* slots, const int* group,
                               const long long* group_begin, int ngroup, long long nitems,
                               unsigned long long* counter, size_t smem, int grid,
                               cudaStream_t s);
cudaError_t launch_batch_decide(SlotDesc* slots, int n, bool f64, cudaStream_t s);
cudaError_t launch_batch_commit(SlotDesc* slots, int n, int maxN, bool f64, cudaStream_t s);
cudaError_t batch_score_occupancy(bool f64, int R, size_t smem, int* blocks_per_sm);
size_t gram_smem_bytes(bool f64, int d, int R);
// Autotuned tile-width cache per (d, ceil log2 N): 0 if not measured yet.
int cached_width(bool f64, int d, int N);
void store_width(bool f64, int d, int N, int R);
int tiles_at_width(int N, int R);

cudaError_t init_kernel_attributes();
cudaError_t init_screen_attributes(int optin_smem);

}  // namespace trstmi
