// The paper's objective on the GPU: the smooth maximum (log-sum-exp)
//   F_{s,delta}(x) = s + delta log sum_{j<k} exp((x_jk - s) / delta),
//   x_jk = |G_jk|^2 of the column-normalised frame Phi of a variable V,
//   s = max x  (arXiv 2207.06374, Sec. "Optimization procedure"),
// and its real gradient in V (dF/dRe V + i dF/dIm V), for `count` frames of
// one shape at once.
//
// The shift by s cancels (F = delta log sum exp(x / delta) identically), so
// dF/dx_jk = w_jk, the softmax weights exp((x_jk - s)/delta) / S; the
// subgradient of the max (Remark on the shift) adds nothing.  With the
// Hermitian Gram G and M = w (.) G (zero diagonal), the gradient in Phi is
// g = 2 Phi M, i.e. for a pair j < k
//   g_k += 2 w_jk G_jk phi_j,   g_j += 2 w_jk conj(G_jk) phi_k,
// and through the column normalisation phi_k = v_k / r_k
//   grad_k = (g_k - phi_k Re(phi_k^* g_k)) / r_k.
//
// Passes (all on the caller's stream, no host synchronisation):
//   1. k_lse_prepare  r_j and the unit columns as [i][column] planes;
//   2. k_lse_max      s = max_{j<k} |G_jk|^2 per frame (tile pass);
//   3. k_lse_tile     per upper-triangle tile (I, J): G, the weights
//                     e_jk = exp((x_jk - s)/delta), M = e (.) G, and the two
//                     products Phi_I M (to block J) and Phi_J M^* (to block
//                     I), written as per-tile partials with the tile's sum
//                     of e (no atomics: the result does not depend on the
//                     order the tiles ran in);
//   4. k_lse_total    S = sum of the tiles' sums in a fixed order, F;
//   5. k_lse_finish   per column: the partials of its tiles in a fixed
//                     order, / S, times 2, projected through the
//                     normalisation.
#include <algorithm>

#include "kernels.h"
#include "tile.cuh"

namespace trstmi {

namespace {

constexpr int kLseThreads = 256;

template <typename T> struct LseArgs {
  int N, d, nb, ntiles, count;
  double delta;
  const double* v;          // count x N x d complex (interleaved), caller's variables
  T* planes;                // count x [d x N re][d x N im] unit columns
  T* rnorm;                 // count x N column norms
  uint32_t* bad;            // count: a zero column was seen
  typename Mu2Bits<T>::type* smax;   // count: s as bits
  T* part;                  // count x ntiles x [2: to I, to J][2: re, im][d][BT]
  double* part_sum;         // count x ntiles
  double* sums;             // count x [F, s, S]
  double* out;              // count x [F, s], the caller's
  double* grad;             // count x N x d complex, or null
};

template <typename T> __device__ __forceinline__ T exp_of(T x);
template <> __device__ __forceinline__ float exp_of<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double exp_of<double>(double x) { return exp(x); }

// 1. one thread per (frame, column): the variable rounded to T, its norm and
// the unit column
template <typename T>
__global__ void k_lse_prepare(const LseArgs<T> a) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)a.count * a.N) return;
  const int slot = (int)(g / a.N), j = (int)(g - (long long)slot * a.N);
  const int d = a.d, N = a.N;
  const double2* col = reinterpret_cast<const double2*>(a.v) + ((size_t)slot * N + j) * d;
  T* pre = a.planes + (size_t)slot * 2 * d * N;
  T* pim = pre + (size_t)d * N;
  T s = T(0);
  for (int i = 0; i < d; ++i) {
    const double2 x = col[i];
    const T re = (T)x.x, im = (T)x.y;
    s = fma(re, re, fma(im, im, s));
  }
  const T r = sqrt(s);
  a.rnorm[(size_t)slot * N + j] = r;
  if (!(s > T(0))) {
    a.bad[slot] = 1u;
    for (int i = 0; i < d; ++i) { pre[(size_t)i * N + j] = T(0); pim[(size_t)i * N + j] = T(0); }
    return;
  }
  for (int i = 0; i < d; ++i) {
    const double2 x = col[i];
    pre[(size_t)i * N + j] = (T)x.x / r;
    pim[(size_t)i * N + j] = (T)x.y / r;
  }
}

// column blocks I and J of a frame's planes into shared memory (d x BT real,
// d x BT imaginary each; block J only off the diagonal), zeros past N
template <typename T, int BT>
__device__ __forceinline__ void load_blocks(const LseArgs<T>& a, int slot, int I, int J, T* sI,
                                            T* sJ) {
  const int d = a.d, N = a.N;
  const T* pre = a.planes + (size_t)slot * 2 * d * N;
  const T* pim = pre + (size_t)d * N;
  for (int blk = 0; blk < (I == J ? 1 : 2); ++blk) {
    const int c0 = (blk == 0 ? I : J) * BT;
    T* ore = blk == 0 ? sI : sJ;
    T* oim = ore + (size_t)d * BT;
    for (int q = threadIdx.x; q < d * BT; q += blockDim.x) {
      const int i = q / BT, loc = q % BT, gj = c0 + loc;
      ore[q] = gj < N ? pre[(size_t)i * N + gj] : T(0);
      oim[q] = gj < N ? pim[(size_t)i * N + gj] : T(0);
    }
  }
}

// 2. s per frame
template <typename T, int R>
__global__ void __launch_bounds__(kLseThreads) k_lse_max(const LseArgs<T> a) {
  constexpr int BT = 16 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[kLseThreads / 32];
  T* sI = reinterpret_cast<T*>(smem_raw);
  T* sJ = sI + (size_t)2 * a.d * BT;
  const long long nitems = (long long)a.count * a.ntiles;
  for (long long w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int slot = (int)(w / a.ntiles);
    int I, J;
    tile_coords((int)(w - (long long)slot * a.ntiles), I, J);
    __syncthreads();
    load_blocks<T, BT>(a, slot, I, J, sI, sJ);
    __syncthreads();
    T m = tile_pairs_max<T, R>(sI, sI + (size_t)a.d * BT, I == J ? sI : sJ, a.d, a.N, I, J,
                               T(-1), nullptr);
    m = block_max<T>(m, red);
    if (threadIdx.x == 0) atomic_max_nonneg(a.smax + slot, m);
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// 3. per tile: weights, M = e (.) G and the two block products
template <typename T, int R>
__global__ void __launch_bounds__(kLseThreads) k_lse_tile(const LseArgs<T> a) {
  constexpr int BT = 16 * R;
  constexpr int MP = BT + 1;                  // padded row pitch of M
  constexpr int STEP = kLseThreads / BT;      // rows i handled side by side
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kLseThreads / 32];
  const int d = a.d, N = a.N;
  T* sI = reinterpret_cast<T*>(smem_raw);
  T* sJ = sI + (size_t)2 * d * BT;
  T* sMre = sJ + (size_t)2 * d * BT;
  T* sMim = sMre + (size_t)BT * MP;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const long long nitems = (long long)a.count * a.ntiles;
  for (long long w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int slot = (int)(w / a.ntiles);
    const int tau = (int)(w - (long long)slot * a.ntiles);
    int I, J;
    tile_coords(tau, I, J);
    const T s = nonneg_from_bits(a.smax[slot]);
    const T delta = (T)a.delta;
    __syncthreads();
    load_blocks<T, BT>(a, slot, I, J, sI, sJ);
    __syncthreads();
    const T* bI = sI;
    const T* bJ = I == J ? sI : sJ;
    // G of the tile, as in the search's tile pass
    MicroTile<T, R> acc;
    acc.zero();
#pragma unroll 2
    for (int i = 0; i < d; ++i) {
      T ar[R], ai[R], br[R], bi[R];
      load_run<T, R>(bI + i * BT + R * ty, ar);
      load_run<T, R>(bI + (size_t)d * BT + i * BT + R * ty, ai);
      load_run<T, R>(bJ + i * BT + R * tx, br);
      load_run<T, R>(bJ + (size_t)d * BT + i * BT + R * tx, bi);
      acc.step(ar, ai, br, bi);
    }
    double esum = 0.0;
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) {
        const int jl = R * ty + x, kl = R * tx + y;
        const int gj = I * BT + jl, gk = J * BT + kl;
        T mre = T(0), mim = T(0);
        if (gj < gk && gk < N) {
          const T gre = acc.get_re(x, y), gim = acc.get_im(x, y);
          const T e = exp_of<T>((pair_abs2(gre, gim) - s) / delta);
          esum += (double)e;
          mre = e * gre;
          mim = e * gim;
        }
        sMre[jl * MP + kl] = mre;
        sMim[jl * MP + kl] = mim;
      }
    esum = block_sum(esum, red);
    if (threadIdx.x == 0) a.part_sum[(size_t)slot * a.ntiles + tau] = esum;
    __syncthreads();
    // Phi_I M -> columns of block J:  P[i][kl] = sum_jl phi_I[i][jl] M[jl][kl]
    // Phi_J M^* -> columns of block I: Q[i][jl] = sum_kl phi_J[i][kl] conj(M[jl][kl])
    T* part = a.part + ((size_t)slot * a.ntiles + tau) * 4 * d * BT;
    const int col = threadIdx.x % BT, i0 = threadIdx.x / BT;
    for (int side = 0; side < 2; ++side) {
      const T* src = side == 0 ? bI : bJ;       // side 0: to J; side 1: to I
      T* dst = part + (size_t)(side == 0 ? 1 : 0) * 2 * d * BT;
      for (int ib = i0; ib < d; ib += 8 * STEP) {
        T pr[8], pi[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { pr[u] = T(0); pi[u] = T(0); }
        for (int l = 0; l < BT; ++l) {
          const T mr = side == 0 ? sMre[l * MP + col] : sMre[col * MP + l];
          const T mi = side == 0 ? sMim[l * MP + col] : -sMim[col * MP + l];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = ib + u * STEP;
            if (i < d) {
              const T re = src[i * BT + l], im = src[(size_t)d * BT + i * BT + l];
              pr[u] = fma(re, mr, fma(-im, mi, pr[u]));
              pi[u] = fma(re, mi, fma(im, mr, pi[u]));
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = ib + u * STEP;
          if (i < d) {
            dst[i * BT + col] = pr[u];
            dst[(size_t)d * BT + i * BT + col] = pi[u];
          }
        }
      }
    }
  }
}

// 4. one CTA per frame: S over the tiles in a fixed order, F = s + delta log S
template <typename T>
__global__ void __launch_bounds__(kLseThreads) k_lse_total(const LseArgs<T> a) {
  __shared__ double red[kLseThreads / 32];
  const int slot = blockIdx.x;
  double v = 0.0;
  for (int tau = threadIdx.x; tau < a.ntiles; tau += blockDim.x)
    v += a.part_sum[(size_t)slot * a.ntiles + tau];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    const double s = (double)nonneg_from_bits(a.smax[slot]);
    double* o = a.sums + 3 * (size_t)slot;
    if (a.bad[slot]) {
      o[0] = o[1] = o[2] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      o[0] = s + a.delta * log(v);
      o[1] = s;
      o[2] = v;
    }
    a.out[2 * (size_t)slot] = o[0];
    a.out[2 * (size_t)slot + 1] = o[1];
  }
}

// 5. one thread per (frame, column): the partials of the column's tiles in a
// fixed order (tiles (I', b) for I' <= b to its block J side, then (b, J')
// for J' >= b to its block I side), 2 / S, then the normalisation
template <typename T, int R>
__global__ void k_lse_finish(const LseArgs<T> a) {
  constexpr int BT = 16 * R;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)a.count * a.N) return;
  const int slot = (int)(g / a.N), j = (int)(g - (long long)slot * a.N);
  const int d = a.d, N = a.N, b = j / BT, loc = j % BT;
  const double* o = a.sums + 3 * (size_t)slot;
  double2* gout = reinterpret_cast<double2*>(a.grad) + ((size_t)slot * N + j) * d;
  if (a.bad[slot]) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int i = 0; i < d; ++i) gout[i] = make_double2(nan, nan);
    return;
  }
  const double scale = 2.0 / o[2];
  const T* part = a.part + (size_t)slot * a.ntiles * 4 * d * BT;
  const T* pre = a.planes + (size_t)slot * 2 * d * N;
  const T* pim = pre + (size_t)d * N;
  double rad = 0.0;
  for (int i = 0; i < d; ++i) {
    double gr = 0.0, gi = 0.0;
    for (int I = 0; I <= b; ++I) {               // tiles (I, b): side "to J"
      const T* p = part + ((size_t)(b * (b + 1) / 2 + I) * 4 + 2) * d * BT;
      gr += (double)p[i * BT + loc];
      gi += (double)p[(size_t)d * BT + i * BT + loc];
    }
    for (int J = b; J < a.nb; ++J) {             // tiles (b, J): side "to I"
      const T* p = part + ((size_t)(J * (J + 1) / 2 + b) * 4 + 0) * d * BT;
      gr += (double)p[i * BT + loc];
      gi += (double)p[(size_t)d * BT + i * BT + loc];
    }
    gr *= scale;
    gi *= scale;
    gout[i] = make_double2(gr, gi);
    rad += (double)pre[(size_t)i * N + j] * gr + (double)pim[(size_t)i * N + j] * gi;
  }
  const double inv_r = 1.0 / (double)a.rnorm[(size_t)slot * N + j];
  for (int i = 0; i < d; ++i) {
    const double2 q = gout[i];
    gout[i] = make_double2((q.x - (double)pre[(size_t)i * N + j] * rad) * inv_r,
                           (q.y - (double)pim[(size_t)i * N + j] * rad) * inv_r);
  }
}

template <typename T> size_t lse_smem(int d, int R) {
  const size_t BT = 16 * (size_t)R;
  return (4 * (size_t)d * BT + 2 * BT * (BT + 1)) * sizeof(T);
}

template <typename T> int lse_pick_R(int N, int d) {
  int R = 4;
  while (R > 1 && 16 * R >= 2 * N) R >>= 1;
  while (R > 1 && lse_smem<T>(d, R) > 200 * 1024) R >>= 1;
  return R;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T> struct LseLayout {
  int R, BT, nb, ntiles;
  size_t o_planes, o_rnorm, o_bad, o_smax, o_part, o_psum, o_out, total;
};

template <typename T> LseLayout<T> lse_layout(int N, int d, int count) {
  LseLayout<T> L;
  L.R = lse_pick_R<T>(N, d);
  L.BT = 16 * L.R;
  L.nb = (N + L.BT - 1) / L.BT;
  L.ntiles = L.nb * (L.nb + 1) / 2;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off = up256(off + bytes); return at; };
  L.o_planes = take((size_t)count * 2 * d * N * sizeof(T));
  L.o_rnorm = take((size_t)count * N * sizeof(T));
  L.o_bad = take((size_t)count * sizeof(uint32_t));
  L.o_smax = take((size_t)count * sizeof(typename Mu2Bits<T>::type));
  L.o_part = take((size_t)count * L.ntiles * 4 * d * L.BT * sizeof(T));
  L.o_psum = take((size_t)count * L.ntiles * sizeof(double));
  L.o_out = take((size_t)count * 3 * sizeof(double));
  L.total = off;
  return L;
}

template <typename K> cudaError_t lse_grid(K kernel, size_t smem, long long items, int num_sms,
                                           int* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLseThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  *grid = (int)std::min<long long>(items, (long long)num_sms * per_sm);
  return cudaSuccess;
}

template <typename T, int R>
cudaError_t lse_launch_R(const LseArgs<T>& a, int num_sms, cudaStream_t s) {
  const size_t smem_max = (size_t)4 * a.d * 16 * R * sizeof(T);
  const size_t smem_tile = lse_smem<T>(a.d, R);
  const long long items = (long long)a.count * a.ntiles;
  int grid = 0;
  cudaError_t e = lse_grid(k_lse_max<T, R>, smem_max, items, num_sms, &grid);
  if (e != cudaSuccess) return e;
  k_lse_max<T, R><<<grid, kLseThreads, smem_max, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = lse_grid(k_lse_tile<T, R>, smem_tile, items, num_sms, &grid)) != cudaSuccess) return e;
  k_lse_tile<T, R><<<grid, kLseThreads, smem_tile, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_lse_total<T><<<a.count, kLseThreads, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.grad) {
    const long long threads = (long long)a.count * a.N;
    k_lse_finish<T, R><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
cudaError_t lse_run(int N, int d, int count, const double* v, double delta, void* scratch,
                    double* out, double* grad, int num_sms, cudaStream_t s) {
  const LseLayout<T> L = lse_layout<T>(N, d, count);
  unsigned char* b = static_cast<unsigned char*>(scratch);
  LseArgs<T> a;
  a.N = N; a.d = d; a.nb = L.nb; a.ntiles = L.ntiles; a.count = count;
  a.delta = delta;
  a.v = v;
  a.planes = reinterpret_cast<T*>(b + L.o_planes);
  a.rnorm = reinterpret_cast<T*>(b + L.o_rnorm);
  a.bad = reinterpret_cast<uint32_t*>(b + L.o_bad);
  a.smax = reinterpret_cast<typename Mu2Bits<T>::type*>(b + L.o_smax);
  a.part = reinterpret_cast<T*>(b + L.o_part);
  a.part_sum = reinterpret_cast<double*>(b + L.o_psum);
  a.sums = reinterpret_cast<double*>(b + L.o_out);
  a.out = out;
  a.grad = grad;
  cudaError_t e;
  // the flags and maxima accumulate; everything else is overwritten
  if ((e = cudaMemsetAsync(b + L.o_bad, 0, L.o_part - L.o_bad, s)) != cudaSuccess) return e;
  const long long threads = (long long)count * N;
  k_lse_prepare<T><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (L.R) {
    case 4: e = lse_launch_R<T, 4>(a, num_sms, s); break;
    case 2: e = lse_launch_R<T, 2>(a, num_sms, s); break;
    default: e = lse_launch_R<T, 1>(a, num_sms, s); break;
  }
  return e;
}

template <typename K> cudaError_t lse_allow(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

}  // namespace

size_t lse_scratch_bytes(int N, int d, int count, bool f64) {
  return f64 ? lse_layout<double>(N, d, count).total : lse_layout<float>(N, d, count).total;
}

cudaError_t launch_lse(int N, int d, int count, const double* v, double delta, bool f64,
                       void* scratch, double* out, double* grad, int num_sms, cudaStream_t s) {
  if (N < 2 || d < 1 || d > kMaxD || count < 1 || !(delta > 0.0)) return cudaErrorInvalidValue;
  return f64 ? lse_run<double>(N, d, count, v, delta, scratch, out, grad, num_sms, s)
             : lse_run<float>(N, d, count, v, delta, scratch, out, grad, num_sms, s);
}

cudaError_t init_lse_attributes(int optin) {
  cudaError_t e;
  if ((e = lse_allow(k_lse_max<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_max<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_max<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_max<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_max<double, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_max<double, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<double, 2>, optin)) != cudaSuccess) return e;
  return lse_allow(k_lse_tile<double, 1>, optin);
}

}  // namespace trstmi
