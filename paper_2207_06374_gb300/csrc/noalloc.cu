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
  uint32_t overflow;
};

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

// Binary32 rounding of the frame into the scratch.
__global__ void k_round_to_f32(size_t n, const double2* in, float2* out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

}  // namespace
}  // namespace trstmi

using namespace trstmi;

extern "C" int trstmi_mu2_frame_noalloc(int N, int d, const double* phi_dev, double* mu2_dev,
                                        void* stream) {
  if (N < 1 || d < 1 || d > kMaxD || !phi_dev || !mu2_dev) return TRSTMI_EINVAL;
  if ((size_t)N * (size_t)d > kNoAllocMaxEntries) return TRSTMI_ESIZE;
  NoAllocScratch* sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc) return rc;
  int num_sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TRSTMI_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)N * d;
  // the array keeps the previous call's contents: clear what accumulates
  if (cudaMemsetAsync(sc->mu2_32, 0, sizeof(sc->mu2_32) + 2 * sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(mu2_dev, 0, sizeof(double), s) != cudaSuccess)
    return TRSTMI_ECUDA;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_round_to_f32<<<grid, 256, 0, s>>>(n, reinterpret_cast<const double2*>(phi_dev), sc->frame32);
  if (cudaGetLastError() != cudaSuccess) return TRSTMI_ECUDA;
  // binary32 max, binary32 preselection of the pairs within its error bound
  // of that max, binary64 over those pairs; full binary64 pass on overflow
  GramSource src{};
  src.perturb = false;
  src.phi = sc->frame32;
  if (launch_gram_f32(N, d, 1, src, &sc->mu2_32[0], nullptr, num_sms, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  const float margin = (float)(8.0 * (2.0 * d + 2.0) / 16777216.0);
  PairFilter pf{&sc->mu2_32[0], margin, sc->pairs, &sc->npairs, kNoAllocPairCap, &sc->overflow};
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
