// Shared device definitions of the TRSTMI CUDA path.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace trstmi {

// Error bits recorded on the device (DevState::error).
enum : uint32_t {
  kErrTimeout = 1u,        // a bounded wait gave up
  kErrZeroColumn = 2u,     // a column had zero norm (cannot be normalised)
};

// Per-instance search state, resident in device memory.  Every kernel of an
// iteration reads it, so the host never synchronises between iterations.
struct DevState {
  double mu2_cur;     // mu^2 of the current frame in the deciding precision
  double delta;       // trust radius for the next iteration
  double delta_used;  // radius of the iteration in progress
  double mu2_best;    // mu^2 of the chosen candidate (deciding precision)
  double mu2_screen;  // its screen / fp32 score
  double target2;     // stop once mu2_cur <= target2 (negative: never)
  double gamma_inc, gamma_dec, delta_min, delta_max;
  double screen_min_delta;  // screen modes: rank with the tensor-core screen only while
                            // delta_used >= this; below it, with the fp32 Gram of all K
  uint32_t use_screen;      // this iteration ranks with the screen
  uint32_t use_full;        // this iteration ranks with the fp32 Gram of every candidate
  uint32_t t;         // iterations completed
  uint32_t t_stop;    // no iteration starts with t >= t_stop
  uint32_t cstar;     // chosen candidate of the iteration in progress
  uint32_t accepted;  // decision of the iteration in progress
  uint32_t accepts;   // accepted candidates so far
  uint32_t done;      // target reached
  uint32_t active;    // the iteration in progress runs (set by its first kernel)
  uint32_t error;     // kErr* bits
  uint32_t npairs;    // certification pair list fill
  uint32_t overflow;  // certification pair list overflowed -> full binary64 pass
  uint32_t trace_cap;
  uint32_t t_call;        // t when the current trstmi_step call started
  uint32_t accepts_call;  // accepts when the current trstmi_step call started
  uint32_t certify;   // screen modes: the best survivor is certified in binary64 (else it
                      // is rejected on its binary32 score, see certify_margin_mu2)
};

// Screen modes: the best survivor's binary32 mu^2 (fp32 generation from the
// binary32 frame, fp32 Gram) and its binary64 mu^2 differ by less than
// 2 (2d + 18) 2^-24 for unit columns: the entries differ by at most 8 ulp
// (frame rounding, fp32 Box-Muller, normalisation), a Gram entry by at most
// (2d + 2) ulp more (its 2d-term dot products), and |G| <= 1.  A survivor whose
// binary32 mu^2 exceeds the current mu^2 by twice that bound is rejected by the
// exact rule as well, so it is rejected without the binary64 certification.
__host__ __device__ inline double certify_margin_mu2(int d) {
  return 4.0 * (2.0 * d + 18.0) * 5.9604644775390625e-8;
}

struct TraceRowDev {
  uint32_t t, cstar;
  double mu2_best, mu2_screen, mu2_cur, delta_used, delta_next;
  int32_t accepted, flags;  // flags bit 0: ranked by the tensor-core screen;
                            // bit 1: rejected on the binary32 bound (no binary64 certification)
};

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Non-negative IEEE values order like their bit patterns as unsigned ints,
// so maxima of |G|^2 are kept with integer atomics.
__device__ __forceinline__ void atomic_max_nonneg(unsigned int* p, float v) {
  atomicMax(p, __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ float nonneg_from_bits(unsigned int b) { return __uint_as_float(b); }
__device__ __forceinline__ double nonneg_from_bits(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

template <typename T> struct Mu2Bits;
template <> struct Mu2Bits<float> { using type = unsigned int; };
template <> struct Mu2Bits<double> { using type = unsigned long long; };

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace trstmi
