// Allocation-free certified coherence of a caller frame in device memory
// (trstmi_mu2_frame_noalloc, include/trstmi.h).
//
// Some callers cannot allocate device memory: their device memory belongs to
// another allocator (a framework's caching allocator) that must not be
// bypassed, or they run in loops where cudaMalloc / cudaFree would stall on
// an implicit device synchronisation.  This entry point therefore keeps all
// of its scratch -- the binary32 copy of the frame, the binary32 maxima, the
// list of preselected pairs and its counters -- in one file-scope static
// device array.  Every GPU that loads the library holds that array until the
// process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "../../include/trstmi.h"
#include "kernels.h"

namespace trstmi {
namespace {

// Limits of the static scratch.
constexpr size_t kNoAllocMaxEntries = 131072;   // N * d complex entries (1 MiB of float2)
constexpr uint32_t kNoAllocPairCap = 65536;     // preselected pairs (512 KiB)

struct NoAllocScratch {
  float2 frame32[kNoAllocMaxEntries];
  uint2 pairs[kNoAllocPairCap];
  unsigned int mu2_32[2];      // binary32 max, and the filter pass's own max
  uint32_t npairs;
  uint32_t overflow;           // also set when the binary32 passes cannot be trusted
  unsigned long long norm2_max;  // binary64 bits of the largest squared column norm
};

// Range of the largest squared column norm M in which the binary32 passes
// are used: within it no |G_jk|^2 <= M^2 overflows binary32, and the scaled
// margin (>= 3e-17) dwarfs the absolute error of underflowed products, so
// every |G| whose binary32 square is subnormal lies inside the kept range.
// Outside it the full binary64 pass decides alone.
constexpr double kNoAllocNormLo = 0x1p-40, kNoAllocNormHi = 0x1p40;

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the array, looked up once per device (host code may not
// use the symbol itself as a device pointer).
std::mutex g_setup_mu;
NoAllocScratch* g_scratch_ptr[64] = {nullptr};

int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TRSTMI_ECUDA;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    if (init_kernel_attributes() != cudaSuccess) return TRSTMI_ECUDA;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TRSTMI_ECUDA;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TRSTMI_OK;
}

// Binary32 rounding of the frame into the scratch, one warp per column, and
// the largest squared column norm (binary64) for the margin of the pair
// filter.  A column norm outside [kNoAllocNormLo, kNoAllocNormHi] (or not
// finite) routes the call to the full binary64 pass.
__global__ void k_round_to_f32(int N, int d, const double2* in, float2* out,
                               unsigned long long* norm2_max, uint32_t* force_full) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < N; j += warps) {
    const double2* col = in + (size_t)j * d;
    float2* o = out + (size_t)j * d;
    double acc = 0.0;
    for (int i = lane; i < d; i += 32) {
      const double2 v = col[i];
      o[i] = make_float2((float)v.x, (float)v.y);
      acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    }
    for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    if (lane == 0) {
      if (!(acc >= kNoAllocNormLo && acc <= kNoAllocNormHi)) *force_full = 1u;
      if (acc >= 0.0) atomicMax(norm2_max, (unsigned long long)__double_as_longlong(acc));
    }
  }
}

}  // namespace
}  // namespace trstmi

using namespace trstmi;

extern "C" int trstmi_mu2_frame_noalloc(int N, int d, const double* phi_dev, double* mu2_dev,
                                        void* stream) {
  if (N < 1 || d < 1 || d > kMaxD || !phi_dev || !mu2_dev) return TRSTMI_EINVAL;
  // the frame is read as 16-byte double2 entries, the result updated by
  // 64-bit atomics
  if (reinterpret_cast<uintptr_t>(phi_dev) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(mu2_dev) % 8 != 0)
    return TRSTMI_EINVAL;
  if ((size_t)N * (size_t)d > kNoAllocMaxEntries) return TRSTMI_ESIZE;
  NoAllocScratch* sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc) return rc;
  int num_sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TRSTMI_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear what accumulates
  // (the two maxima, the pair count, the overflow flag and the norm maximum
  // are contiguous)
  static_assert(offsetof(NoAllocScratch, norm2_max) ==
                    offsetof(NoAllocScratch, mu2_32) + 2 * sizeof(unsigned int) + 2 * sizeof(uint32_t),
                "cleared span");
  if (cudaMemsetAsync(sc->mu2_32, 0,
                      offsetof(NoAllocScratch, norm2_max) + sizeof(unsigned long long) -
                          offsetof(NoAllocScratch, mu2_32),
                      s) != cudaSuccess ||
      cudaMemsetAsync(mu2_dev, 0, sizeof(double), s) != cudaSuccess)
    return TRSTMI_ECUDA;
  const int grid = std::min((N + 7) / 8, 4096);
  k_round_to_f32<<<grid, 256, 0, s>>>(N, d, reinterpret_cast<const double2*>(phi_dev),
                                      sc->frame32, &sc->norm2_max, &sc->overflow);
  if (cudaGetLastError() != cudaSuccess) return TRSTMI_ECUDA;
  // binary32 max, binary32 preselection of the pairs within its error bound
  // of that max, binary64 over those pairs; full binary64 pass on overflow
  GramSource src{};
  src.perturb = false;
  src.phi = sc->frame32;
  if (launch_gram_f32(N, d, 1, src, &sc->mu2_32[0], nullptr, num_sms, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  // the binary32 error of |G_jk| is bounded by the unit-column bound times
  // |phi_j| |phi_k| <= max_j |phi_j|^2, so the margin is scaled by that
  const float margin = (float)(8.0 * (2.0 * d + 2.0) / 16777216.0);
  PairFilter pf{&sc->mu2_32[0], margin, sc->pairs, &sc->npairs, kNoAllocPairCap, &sc->overflow,
                &sc->norm2_max};
  if (launch_gram_f32(N, d, 1, src, &sc->mu2_32[1], &pf, num_sms, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  unsigned long long* out = reinterpret_cast<unsigned long long*>(mu2_dev);
  if (launch_pairs64(nullptr, &sc->npairs, sc->pairs, kNoAllocPairCap, d,
                     reinterpret_cast<const double2*>(phi_dev), out, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  GramSource full{};
  full.perturb = false;
  full.phi = phi_dev;
  full.gate = &sc->overflow;
  if (launch_gram_f64(N, d, 1, full, out, num_sms, s) != cudaSuccess) return TRSTMI_ECUDA;
  return TRSTMI_OK;
}
