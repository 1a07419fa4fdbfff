// Measured arithmetic peaks of the GPU (trstmi_measure_peaks, include/trstmi.h):
// the denominators of the binary32, binary64 and tf32 rooflines.
//
// Each rate comes from a short loop that keeps one unit busy on every SM:
//   - FFMA / DFMA: 32 warps per SM, each thread eight independent fused
//     multiply-add chains (2 flops each);
//   - bf16 and tf32 tensor cores: one CTA per SM whose elected thread issues
//     back-to-back tcgen05.mma of M = 128, N = 256 (K = 16 bf16 or 8 tf32 per
//     instruction) from shared-memory operands into tensor memory.
// Launches are timed with CUDA events on the caller's stream after a warm-up
// launch.  Operands hold small nonzero values so that the units switch as in
// real work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/trstmi.h"
#include "kernels.h"

namespace trstmi {
namespace {

constexpr int kPeakChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T seed, T* sink) {
  T a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed + (T)(threadIdx.x + c) * (T)1e-7;
  const T m = (T)0.999999, b = (T)1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = fma(a[c], m, b);
    }
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += a[c];
  if (s == (T)-1) sink[blockIdx.x] = s;   // never true; keeps the chains alive
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// kind: 0 = bf16 (kind::f16, K = 16), 1 = tf32 (kind::tf32, K = 8); both read
// 32 bytes of K per row per instruction.  *status: 1 if a completion wait ran
// out of time (2 s), which the host reports as a timeout.
template <int kKind>
__global__ void __launch_bounds__(128) k_mma_loop(int iters, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char raw[];
  __shared__ unsigned long long bar;
  __shared__ uint32_t tbase;
  const uint32_t r0 = smem_addr(raw);
  unsigned char* sm = raw + (((r0 + 1023u) & ~1023u) - r0);
  const uint32_t base = smem_addr(sm);
  // A: 128 rows x 128 B; B: 256 rows x 128 B; values +-0.5 (bf16 pairs or fp32)
  uint32_t* w = reinterpret_cast<uint32_t*>(sm);
  for (int i = threadIdx.x; i < (16384 + 32768) / 4; i += blockDim.x) {
    const bool neg = ((i * 2654435761u) >> 13) & 1u;
    w[i] = kKind == 0 ? (neg ? 0xBF00BF00u : 0x3F003F00u) : (neg ? 0xBF000000u : 0x3F000000u);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     smem_addr(&tbase))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = tbase;
  if (threadIdx.x == 0) {
    // K-major, 128-byte swizzle, 1024-byte stride between 8-row groups
    const uint32_t hi = (1024u >> 4) | (1u << 14) | (2u << 29);
    const uint32_t alo = ((base >> 4) & 0x3FFFu) | (1u << 16);
    const uint32_t blo = (((base + 16384u) >> 4) & 0x3FFFu) | (1u << 16);
    const uint32_t fmt = kKind == 0 ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) |
                           ((128u >> 4) << 24);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) {
        const uint32_t acc = (i | k) ? 1u : 0u;
        if (kKind == 0)
          asm volatile(
              "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %4, 0;\n"
              " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %5};\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(tm),
              "r"(alo + 2u * k), "r"(blo + 2u * k), "r"(idesc), "r"(acc), "r"(hi)
              : "memory");
        else
          asm volatile(
              "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %4, 0;\n"
              " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %5};\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %3, p;\n}\n" ::"r"(tm),
              "r"(alo + 2u * k), "r"(blo + 2u * k), "r"(idesc), "r"(acc), "r"(hi)
              : "memory");
      }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&bar))
        : "memory");
    // bounded wait for the MMAs to complete
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    uint32_t ok = 0;
    while (!ok) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, 1000000;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_addr(&bar))
          : "memory");
      unsigned long long t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if (!ok && t1 - t0 > 2000000000ull) { atomicExch(status, 1u); break; }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tm) : "memory");
}

// operands use 49 KiB; asking for 120 KiB keeps the loop at one CTA per SM
constexpr size_t kMmaSmem = 120 * 1024;

// Milliseconds of `launch` (after one warm-up), timed with events on s.
template <class F> cudaError_t time_ms(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace trstmi

using namespace trstmi;

extern "C" int trstmi_measure_peaks(trstmi_peaks* out, void* stream) {
  if (!out) return TRSTMI_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TRSTMI_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, 64 * 1024) != cudaSuccess) { cudaGetLastError(); return TRSTMI_ENOMEM; }
  uint32_t* status = static_cast<uint32_t*>(scratch);
  int rc = TRSTMI_OK;
  float ms = 0.f;
  do {
    if (cudaMemsetAsync(status, 0, sizeof(uint32_t), s) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    // FFMA: 4 CTAs of 256 threads per SM (32 warps), 8 chains x 16 per iteration
    const int fgrid = 4 * sms, fiters = 4096;
    if (time_ms([&] {
          k_fma_loop<float><<<fgrid, 256, 0, s>>>(fiters, 1.0f,
                                                  reinterpret_cast<float*>(status) + 16);
          return cudaGetLastError();
        }, s, &ms) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    out->fp32_tflops = 2.0 * kPeakChains * 16.0 * fiters * fgrid * 256.0 / (ms * 1e-3) / 1e12;
    const int diters = 256;
    if (time_ms([&] {
          k_fma_loop<double><<<fgrid, 256, 0, s>>>(diters, 1.0,
                                                   reinterpret_cast<double*>(status) + 16);
          return cudaGetLastError();
        }, s, &ms) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    out->fp64_tflops = 2.0 * kPeakChains * 16.0 * diters * fgrid * 256.0 / (ms * 1e-3) / 1e12;
    // tensor cores: one CTA per SM
    const int miters = 16384;
    if (cudaFuncSetAttribute(k_mma_loop<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMmaSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_mma_loop<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMmaSmem) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    if (time_ms([&] {
          k_mma_loop<0><<<sms, 128, kMmaSmem, s>>>(miters, status);
          return cudaGetLastError();
        }, s, &ms) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    out->bf16_tflops = 2.0 * 128 * 256 * 16 * 4.0 * miters * sms / (ms * 1e-3) / 1e12;
    if (time_ms([&] {
          k_mma_loop<1><<<sms, 128, kMmaSmem, s>>>(miters / 2, status);
          return cudaGetLastError();
        }, s, &ms) != cudaSuccess) { rc = TRSTMI_ECUDA; break; }
    out->tf32_tflops = 2.0 * 128 * 256 * 8 * 4.0 * (miters / 2) * sms / (ms * 1e-3) / 1e12;
    uint32_t st = 0;
    if (cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = TRSTMI_ECUDA;
      break;
    }
    if (st) rc = TRSTMI_ETIMEOUT;
  } while (0);
  if (rc == TRSTMI_ECUDA) cudaGetLastError();
  cudaFree(scratch);
  return rc;
}
