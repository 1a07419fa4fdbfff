// Frame certificates on the GPU (binary64): the largest and smallest
// off-diagonal |G_jk| of the column-normalised frame and the number of
// distinct distances among them, for the bounds and observations of arXiv
// 2207.06374, Sec. "Conjectures from Numerics" (orthoplex and Levenshtein
// bounds; the single-distance observation) and the chordal distance
// sqrt(1 - |<x, y>|^2) of Sec. "Introduction".
//
// Distinct distances at resolution tol: every value v = |G_jk| marks bin
// floor(v / tol) in a bitmap; one distance is a maximal run of consecutive
// marked bins (values closer than tol always share a run, values farther
// apart than 2 tol never do).
//
// Passes: k_diag_prepare (unit columns as [i][column] planes), k_diag_tile
// (per upper-triangle tile: G by the search's micro-tile arithmetic, max and
// min of |G|^2, bitmap marks), k_diag_runs (run starts counted per bitmap
// word).
#include <algorithm>

#include "kernels.h"
#include "tile.cuh"

namespace trstmi {

namespace {

constexpr int kDiagThreads = 256;

struct DiagArgs {
  int N, d, nb, ntiles;
  const double* v;             // N x d complex (interleaved), the frame as given
  double* planes;              // [d x N re][d x N im] unit columns
  unsigned long long* mx;      // max |G|^2 (bits)
  unsigned long long* mn;      // min |G|^2 (bits)
  uint32_t* runs;              // distinct distances
  uint32_t* bad;               // a zero column was seen
  uint32_t* bits;              // nbins bits
  long long nbins;
  double tol;
};

__global__ void k_diag_prepare(const DiagArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  const int d = a.d, N = a.N;
  const double2* col = reinterpret_cast<const double2*>(a.v) + (size_t)j * d;
  double* pre = a.planes;
  double* pim = pre + (size_t)d * N;
  double s = 0.0;
  for (int i = 0; i < d; ++i) {
    const double2 x = col[i];
    s = fma(x.x, x.x, fma(x.y, x.y, s));
  }
  if (!(s > 0.0)) {
    *a.bad = 1u;
    for (int i = 0; i < d; ++i) { pre[(size_t)i * N + j] = 0.0; pim[(size_t)i * N + j] = 0.0; }
    return;
  }
  const double r = sqrt(s);
  for (int i = 0; i < d; ++i) {
    const double2 x = col[i];
    pre[(size_t)i * N + j] = x.x / r;
    pim[(size_t)i * N + j] = x.y / r;
  }
}

// CTA minimum (valid in thread 0); idle slots hold +inf
__device__ __forceinline__ double block_min(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

template <int R>
__global__ void __launch_bounds__(kDiagThreads) k_diag_tile(const DiagArgs a) {
  constexpr int BT = 16 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kDiagThreads / 32];
  const int d = a.d, N = a.N;
  double* sI = reinterpret_cast<double*>(smem_raw);
  double* sJ = sI + (size_t)2 * d * BT;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int tau = blockIdx.x; tau < a.ntiles; tau += gridDim.x) {
    int I, J;
    tile_coords(tau, I, J);
    __syncthreads();
    prefetch_blocks<double, BT>(a.planes, d, N, I, J, sI, false);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const double* bJ = I == J ? sI : sJ;
    MicroTile<double, R> acc;
    acc.zero();
    for (int i = 0; i < d; ++i) {
      double ar[R], ai[R], br[R], bi[R];
      load_run<double, R>(sI + i * BT + R * ty, ar);
      load_run<double, R>(sI + (size_t)d * BT + i * BT + R * ty, ai);
      load_run<double, R>(bJ + i * BT + R * tx, br);
      load_run<double, R>(bJ + (size_t)d * BT + i * BT + R * tx, bi);
      acc.step(ar, ai, br, bi);
    }
    double hi = 0.0, lo = 2.0;
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) {
        const int gj = I * BT + R * ty + x, gk = J * BT + R * tx + y;
        if (gj < gk && gk < N) {
          const double g2 = pair_abs2(acc.get_re(x, y), acc.get_im(x, y));
          hi = fmax(hi, g2);
          lo = fmin(lo, g2);
          long long bin = (long long)floor(sqrt(g2) / a.tol);
          bin = bin < a.nbins ? bin : a.nbins - 1;
          atomicOr(a.bits + (bin >> 5), 1u << (bin & 31));
        }
      }
    hi = block_max<double>(hi, red);
    if (threadIdx.x == 0) atomicMax(a.mx, (unsigned long long)__double_as_longlong(hi));
    lo = block_min(lo, red);
    if (threadIdx.x == 0 && lo <= 1.5)
      atomicMin(a.mn, (unsigned long long)__double_as_longlong(lo));
  }
}

__global__ void k_diag_runs(const DiagArgs a) {
  const long long nwords = (a.nbins + 31) >> 5;
  const long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (w >= nwords) return;
  const uint32_t cur = a.bits[w];
  const uint32_t carry = w > 0 ? (a.bits[w - 1] >> 31) : 0u;   // bin just below this word
  const uint32_t starts = cur & ~((cur << 1) | carry);
  if (starts) atomicAdd(a.runs, (uint32_t)__popc(starts));
}

int diag_R(int N, int d) {
  int R = 4;
  while (R > 1 && 16 * R >= 2 * N) R >>= 1;
  while (R > 1 && (size_t)4 * d * 16 * R * sizeof(double) > 200 * 1024) R >>= 1;
  return R;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t diag_scratch_bytes(int N, int d, double tol) {
  const long long nbins = (long long)std::floor(1.0 / tol) + 2;
  return 256 + up256((size_t)2 * d * N * sizeof(double)) + up256((size_t)((nbins + 31) / 32) * 4);
}

cudaError_t launch_diagnostics(int N, int d, const double* v_dev, double tol, void* scratch,
                               int num_sms, cudaStream_t s) {
  if (N < 2 || d < 1 || d > kMaxD || !(tol >= 1e-7 && tol <= 1.0)) return cudaErrorInvalidValue;
  unsigned char* b = static_cast<unsigned char*>(scratch);
  DiagArgs a;
  a.N = N; a.d = d;
  const int R = diag_R(N, d), BT = 16 * R;
  a.nb = (N + BT - 1) / BT;
  a.ntiles = a.nb * (a.nb + 1) / 2;
  a.v = v_dev;
  a.mx = reinterpret_cast<unsigned long long*>(b);
  a.mn = reinterpret_cast<unsigned long long*>(b + 8);
  a.runs = reinterpret_cast<uint32_t*>(b + 16);
  a.bad = reinterpret_cast<uint32_t*>(b + 20);
  a.planes = reinterpret_cast<double*>(b + 256);
  a.bits = reinterpret_cast<uint32_t*>(b + 256 + up256((size_t)2 * d * N * sizeof(double)));
  a.nbins = (long long)std::floor(1.0 / tol) + 2;
  a.tol = tol;
  const size_t nwords = (size_t)((a.nbins + 31) / 32);
  cudaError_t e;
  if ((e = cudaMemsetAsync(b, 0, 24, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b + 8, 0xff, 8, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.bits, 0, nwords * 4, s)) != cudaSuccess) return e;
  k_diag_prepare<<<(N + 127) / 128, 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = (size_t)4 * d * BT * sizeof(double);
  const int grid = std::min(a.ntiles, num_sms * 2);
  switch (R) {
    case 4: k_diag_tile<4><<<grid, kDiagThreads, smem, s>>>(a); break;
    case 2: k_diag_tile<2><<<grid, kDiagThreads, smem, s>>>(a); break;
    default: k_diag_tile<1><<<grid, kDiagThreads, smem, s>>>(a); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_diag_runs<<<(unsigned)((nwords + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t init_diag_attributes(int optin) {
  cudaError_t e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, k_diag_tile<4>)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_diag_tile<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncGetAttributes(&fa, k_diag_tile<2>)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_diag_tile<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncGetAttributes(&fa, k_diag_tile<1>)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_diag_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

}  // namespace trstmi
