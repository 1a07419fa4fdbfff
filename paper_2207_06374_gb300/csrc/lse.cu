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
//   2. the search's Gram pass over the planes: s = max_{j<k} |G_jk|^2 per
//                     frame (the same micro-tile arithmetic as below, so
//                     every x_jk has the same bits in both passes);
//   3. k_lse_tile     per upper-triangle tile (I, J), the next tile's column
//                     blocks copied asynchronously meanwhile: G, the weights
//                     e_jk = exp((x_jk - s)/delta), M = e (.) G, and the two
//                     products Phi_I M (to block J) and Phi_J M^* (to block
//                     I), written as per-tile partials with the tile's sum
//                     of e (no atomics: the result does not depend on the
//                     order the tiles ran in);
//   4. k_lse_total    S = sum of the tiles' sums in a fixed order, F;
//   5. k_lse_finish   per group of columns: the partials of each column's
//                     tiles in a fixed order, / S, times 2, staged in shared
//                     memory, projected through the normalisation and
//                     written column by column.
#include <algorithm>

#include "kernels.h"
#include "tile.cuh"

namespace trstmi {

namespace {

constexpr int kLseThreads = 256;

template <typename T> struct LseArgs {
  int N, d, nb, ntiles, count;
  double delta;
  const double* deltas;     // count smoothing parameters (device), or null: delta for all
  const double* v;          // count x N x d complex (interleaved), caller's variables
  T* planes;                // count x [d x N re][d x N im] unit columns
  T* rnorm;                 // count x N column norms
  uint32_t* bad;            // count: a zero column was seen
  int vec;                  // planes copied in 16-byte runs (N % (16 / sizeof(T)) == 0)
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

// R consecutive values to shared or global memory (R * sizeof(T)-aligned)
template <typename T, int R>
__device__ __forceinline__ void store_run(T* p, const T (&v)[R]) {
  if constexpr (sizeof(T) == 4 && R == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (sizeof(T) == 4 && R == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (sizeof(T) == 8 && R % 2 == 0) {
#pragma unroll
    for (int h = 0; h < R; h += 2) *reinterpret_cast<double2*>(p + h) = make_double2(v[h], v[h + 1]);
  } else {
#pragma unroll
    for (int x = 0; x < R; ++x) p[x] = v[x];
  }
}

// Four complex multiply-adds p[c] += (a + ib) (mr[c] + i mi[c]); binary32
// pairs neighbouring columns in paired fused multiply-adds.
template <typename T>
__device__ __forceinline__ void cmac4(T (&pr)[4], T (&pi)[4], T a, T b, const T (&mr)[4],
                                      const T (&mi)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float2 aa = make_float2(a, a), bb = make_float2(b, b), nb = make_float2(-b, -b);
#pragma unroll
    for (int h = 0; h < 4; h += 2) {
      const float2 r = make_float2(mr[h], mr[h + 1]), q = make_float2(mi[h], mi[h + 1]);
      float2 xr = make_float2(pr[h], pr[h + 1]), xi = make_float2(pi[h], pi[h + 1]);
      xr = __ffma2_rn(aa, r, __ffma2_rn(nb, q, xr));
      xi = __ffma2_rn(aa, q, __ffma2_rn(bb, r, xi));
      pr[h] = xr.x; pr[h + 1] = xr.y;
      pi[h] = xi.x; pi[h + 1] = xi.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pr[c] = fma(a, mr[c], fma(-b, mi[c], pr[c]));
      pi[c] = fma(a, mi[c], fma(b, mr[c], pi[c]));
    }
  }
}

// out[i][c] = sum_l src[i][l] X[l][c] over a tile's BT columns: src is a
// column block in shared memory (d x BT real, then d x BT imaginary), X a
// complex BT x BT matrix in shared memory (real and imaginary planes, row
// pitch P), out d x BT real then imaginary (global).  Each thread owns four
// adjacent columns c of two rows i (i0, i0 + RG): per step l one vector load
// of X's row segment per plane and four scalar loads of src, 32 fused
// multiply-adds.
template <typename T, int BT, int P>
__device__ __forceinline__ void block_product(const T* src, const T* xre, const T* xim, T* out,
                                              int d) {
  constexpr int CG = BT / 4;
  constexpr int RG = kLseThreads / CG;
  const int cg = threadIdx.x % CG, rg = threadIdx.x / CG;
  const T* sre = src;
  const T* sim = src + (size_t)d * BT;
  for (int i0 = rg; i0 < d; i0 += 2 * RG) {
    const int i1 = i0 + RG;
    const bool two = i1 < d;
    T pr0[4], pi0[4], pr1[4], pi1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { pr0[c] = pi0[c] = pr1[c] = pi1[c] = T(0); }
#pragma unroll 4
    for (int l = 0; l < BT; ++l) {
      T mr[4], mi[4];
      load_run<T, 4>(xre + l * P + 4 * cg, mr);
      load_run<T, 4>(xim + l * P + 4 * cg, mi);
      const T a0 = sre[i0 * BT + l], b0 = sim[i0 * BT + l];
      const T a1 = two ? sre[i1 * BT + l] : T(0), b1 = two ? sim[i1 * BT + l] : T(0);
      cmac4<T>(pr0, pi0, a0, b0, mr, mi);
      cmac4<T>(pr1, pi1, a1, b1, mr, mi);
    }
    store_run<T, 4>(out + i0 * BT + 4 * cg, pr0);
    store_run<T, 4>(out + (size_t)d * BT + i0 * BT + 4 * cg, pi0);
    if (two) {
      store_run<T, 4>(out + i1 * BT + 4 * cg, pr1);
      store_run<T, 4>(out + (size_t)d * BT + i1 * BT + 4 * cg, pi1);
    }
  }
}

// 3. per tile: weights, M = e (.) G and the two block products.  The
// thread that forms G_jk for its R x R micro-tile keeps M_jk in registers:
// it writes M for Phi_I M (to block J), then M^* transposed for Phi_J M^*
// (to block I), so both products read row segments of one matrix.
template <typename T, int R>
__device__ __forceinline__ void lse_prefetch(const LseArgs<T>& a, long long w, T* dst) {
  const int slot = (int)(w / a.ntiles);
  int I, J;
  tile_coords((int)(w - (long long)slot * a.ntiles), I, J);
  prefetch_blocks<T, 16 * R>(a.planes + (size_t)slot * 2 * a.d * a.N, a.d, a.N, I, J, dst,
                             a.vec != 0);
}

template <typename T, int R>
__global__ void __launch_bounds__(kLseThreads) k_lse_tile(const LseArgs<T> a) {
  constexpr int BT = 16 * R;
  constexpr int P = BT + 4;                   // row pitch of M (vector-aligned)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kLseThreads / 32];
  const int d = a.d, N = a.N;
  // two stages of column blocks (I then J, 4 d BT values each), then M
  T* stage0 = reinterpret_cast<T*>(smem_raw);
  const size_t stage = (size_t)4 * d * BT;
  T* sMre = stage0 + 2 * stage;
  T* sMim = sMre + (size_t)BT * P;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const long long nitems = (long long)a.count * a.ntiles;
  long long w = blockIdx.x;
  if (w < nitems) lse_prefetch<T, R>(a, w, stage0);
  cp_async_commit();
  for (int sg = 0; w < nitems; w += gridDim.x, sg ^= 1) {
    const long long wn = w + gridDim.x;
    if (wn < nitems) lse_prefetch<T, R>(a, wn, stage0 + (sg ^ 1) * stage);
    cp_async_commit();
    cp_async_wait<1>();   // this thread's copies of item w have landed ...
    __syncthreads();      // ... and every other thread's
    const int slot = (int)(w / a.ntiles);
    const int tau = (int)(w - (long long)slot * a.ntiles);
    int I, J;
    tile_coords(tau, I, J);
    const T s = nonneg_from_bits(a.smax[slot]);
    const T delta = (T)(a.deltas ? a.deltas[slot] : a.delta);
    const T* bI = stage0 + sg * stage;
    const T* bJ = I == J ? bI : bI + (size_t)2 * d * BT;
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
    // weights and M (zero outside j < k < N); the thread's few weights are
    // summed in T, the CTA's sum and everything after it in binary64
    T esum = T(0);
    T mre[R][R], mim[R][R];
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) {
        const int gj = I * BT + R * ty + x, gk = J * BT + R * tx + y;
        mre[x][y] = mim[x][y] = T(0);
        if (gj < gk && gk < N) {
          const T gre = acc.get_re(x, y), gim = acc.get_im(x, y);
          const T e = exp_of<T>((pair_abs2(gre, gim) - s) / delta);
          esum += e;
          mre[x][y] = e * gre;
          mim[x][y] = e * gim;
        }
      }
#pragma unroll
    for (int x = 0; x < R; ++x) {
      store_run<T, R>(sMre + (R * ty + x) * P + R * tx, mre[x]);
      store_run<T, R>(sMim + (R * ty + x) * P + R * tx, mim[x]);
    }
    const double tsum = block_sum((double)esum, red);   // its barriers also publish M
    if (threadIdx.x == 0) a.part_sum[(size_t)slot * a.ntiles + tau] = tsum;
    T* part = a.part + ((size_t)slot * a.ntiles + tau) * 4 * d * BT;
    // Phi_I M -> columns of block J:  P[i][kl] = sum_jl phi_I[i][jl] M[jl][kl]
    block_product<T, BT, P>(bI, sMre, sMim, part + (size_t)2 * d * BT, d);
    __syncthreads();
    // Phi_J M^* -> columns of block I: Q[i][jl] = sum_kl phi_J[i][kl] conj(M[jl][kl])
#pragma unroll
    for (int y = 0; y < R; ++y) {
      T cr[R], ci[R];
#pragma unroll
      for (int x = 0; x < R; ++x) { cr[x] = mre[x][y]; ci[x] = -mim[x][y]; }
      store_run<T, R>(sMre + (R * tx + y) * P + R * ty, cr);
      store_run<T, R>(sMim + (R * tx + y) * P + R * ty, ci);
    }
    __syncthreads();
    block_product<T, BT, P>(bJ, sMre, sMim, part, d);
    __syncthreads();      // stage sg and M are free for the next round
  }
  cp_async_wait<0>();
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
      o[0] = s + (a.deltas ? a.deltas[slot] : a.delta) * log(v);
      o[1] = s;
      o[2] = v;
    }
    a.out[2 * (size_t)slot] = o[0];
    a.out[2 * (size_t)slot + 1] = o[1];
  }
}

// 5. one CTA per (frame, group of CW columns).  Thread (row, col) sums, for
// rows i = row, row + 256/CW, ..., the partials of column j = j0 + col over
// its tiles in a fixed order (tiles (I', b) for I' <= b: the side "to J";
// then (b, J') for J' >= b: the side "to I"; b = j / BT), reading runs of
// consecutive columns, and stages 2 g / S and the unit column in shared
// memory; then each warp takes whole columns: Re(phi^* g) by a warp sum and
// the projected, rescaled column written in consecutive entries.
template <typename T, int R>
__global__ void __launch_bounds__(kLseThreads) k_lse_finish(const LseArgs<T> a, int CW) {
  constexpr int BT = 16 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = a.d, N = a.N;
  double2* sG = reinterpret_cast<double2*>(smem_raw);                 // d x CW
  typename Cplx<T>::type* sP = reinterpret_cast<typename Cplx<T>::type*>(sG + (size_t)d * CW);
  const int groups = (N + CW - 1) / CW;
  const int slot = blockIdx.x / groups, j0 = (blockIdx.x - slot * groups) * CW;
  const double* o = a.sums + 3 * (size_t)slot;
  double2* gout = reinterpret_cast<double2*>(a.grad) + (size_t)slot * N * d;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (a.bad[slot]) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int c = warp; c < CW && j0 + c < N; c += kLseThreads / 32)
      for (int i = lane; i < d; i += 32) gout[(size_t)(j0 + c) * d + i] = make_double2(nan, nan);
    return;
  }
  const double scale = 2.0 / o[2];
  const T* part = a.part + (size_t)slot * a.ntiles * 4 * d * BT;
  const T* pre = a.planes + (size_t)slot * 2 * d * N;
  const T* pim = pre + (size_t)d * N;
  {
    const int col = threadIdx.x % CW, row = threadIdx.x / CW, rows = kLseThreads / CW;
    const int j = j0 + col;
    const bool in = j < N;
    const int b = j / BT, loc = j % BT;
    for (int i = row; i < d; i += rows) {
      // summed in T: binary64 arithmetic runs at a small fraction of the
      // binary32 rate, and the partials are T already
      T gr = T(0), gi = T(0);
      if (in) {
#pragma unroll 4
        for (int I = 0; I <= b; ++I) {               // tiles (I, b): side "to J"
          const T* p = part + ((size_t)(b * (b + 1) / 2 + I) * 4 + 2) * d * BT;
          gr += p[i * BT + loc];
          gi += p[(size_t)d * BT + i * BT + loc];
        }
#pragma unroll 4
        for (int J = b; J < a.nb; ++J) {             // tiles (b, J): side "to I"
          const T* p = part + ((size_t)(J * (J + 1) / 2 + b) * 4 + 0) * d * BT;
          gr += p[i * BT + loc];
          gi += p[(size_t)d * BT + i * BT + loc];
        }
      }
      sG[i * CW + col] = make_double2((double)gr * scale, (double)gi * scale);
      typename Cplx<T>::type ph;
      ph.x = in ? pre[(size_t)i * N + j] : T(0);
      ph.y = in ? pim[(size_t)i * N + j] : T(0);
      sP[i * CW + col] = ph;
    }
  }
  __syncthreads();
  for (int c = warp; c < CW; c += kLseThreads / 32) {
    const int j = j0 + c;
    if (j >= N) break;
    double rad = 0.0;
    for (int i = lane; i < d; i += 32) {
      const double2 g = sG[i * CW + c];
      const auto ph = sP[i * CW + c];
      rad += (double)ph.x * g.x + (double)ph.y * g.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rad += __shfl_xor_sync(0xffffffffu, rad, off);
    const double inv_r = 1.0 / (double)a.rnorm[(size_t)slot * N + j];
    for (int i = lane; i < d; i += 32) {
      const double2 g = sG[i * CW + c];
      const auto ph = sP[i * CW + c];
      gout[(size_t)j * d + i] =
          make_double2((g.x - (double)ph.x * rad) * inv_r, (g.y - (double)ph.y * rad) * inv_r);
    }
  }
}

// 5'. The same pass with one CTA per (frame, column block b): thread (row, c4)
// sums four adjacent columns 4 c4 .. 4 c4 + 3 of row i over the block's tiles
// in the same fixed order with vector loads, stages them with the block's
// unit columns, and every warp then finishes whole columns as in k_lse_finish.
// Used while d x BT staged values fit 96 KiB.
template <typename T, int R>
__global__ void __launch_bounds__(kLseThreads) k_lse_finish_block(const LseArgs<T> a) {
  constexpr int BT = 16 * R, C4 = BT / 4, ROWS = kLseThreads / C4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = a.d, N = a.N;
  double2* sG = reinterpret_cast<double2*>(smem_raw);                 // d x BT
  typename Cplx<T>::type* sP = reinterpret_cast<typename Cplx<T>::type*>(sG + (size_t)d * BT);
  const int slot = blockIdx.x / a.nb, b = blockIdx.x - slot * a.nb, j0 = b * BT;
  const double* o = a.sums + 3 * (size_t)slot;
  double2* gout = reinterpret_cast<double2*>(a.grad) + (size_t)slot * N * d;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (a.bad[slot]) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int c = warp; c < BT && j0 + c < N; c += kLseThreads / 32)
      for (int i = lane; i < d; i += 32) gout[(size_t)(j0 + c) * d + i] = make_double2(nan, nan);
    return;
  }
  const double scale = 2.0 / o[2];
  const T* part = a.part + (size_t)slot * a.ntiles * 4 * d * BT;
  const T* pre = a.planes + (size_t)slot * 2 * d * N;
  const T* pim = pre + (size_t)d * N;
  const int c4 = threadIdx.x % C4, row = threadIdx.x / C4;
  for (int i = row; i < d; i += ROWS) {
    T gr[4] = {T(0), T(0), T(0), T(0)}, gi[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 2
    for (int I = 0; I <= b; ++I) {               // tiles (I, b): side "to J"
      const T* p = part + ((size_t)(b * (b + 1) / 2 + I) * 4 + 2) * d * BT + i * BT + 4 * c4;
      T vr[4], vi[4];
      load_run<T, 4>(p, vr);
      load_run<T, 4>(p + (size_t)d * BT, vi);
#pragma unroll
      for (int e = 0; e < 4; ++e) { gr[e] += vr[e]; gi[e] += vi[e]; }
    }
#pragma unroll 2
    for (int J = b; J < a.nb; ++J) {             // tiles (b, J): side "to I"
      const T* p = part + ((size_t)(J * (J + 1) / 2 + b) * 4 + 0) * d * BT + i * BT + 4 * c4;
      T vr[4], vi[4];
      load_run<T, 4>(p, vr);
      load_run<T, 4>(p + (size_t)d * BT, vi);
#pragma unroll
      for (int e = 0; e < 4; ++e) { gr[e] += vr[e]; gi[e] += vi[e]; }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int loc = 4 * c4 + e, j = j0 + loc;
      sG[i * BT + loc] = make_double2((double)gr[e] * scale, (double)gi[e] * scale);
      typename Cplx<T>::type ph;
      ph.x = j < N ? pre[(size_t)i * N + j] : T(0);
      ph.y = j < N ? pim[(size_t)i * N + j] : T(0);
      sP[i * BT + loc] = ph;
    }
  }
  __syncthreads();
  for (int c = warp; c < BT; c += kLseThreads / 32) {
    const int j = j0 + c;
    if (j >= N) break;
    double rad = 0.0;
    for (int i = lane; i < d; i += 32) {
      const double2 g = sG[i * BT + c];
      const auto ph = sP[i * BT + c];
      rad += (double)ph.x * g.x + (double)ph.y * g.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rad += __shfl_xor_sync(0xffffffffu, rad, off);
    const double inv_r = 1.0 / (double)a.rnorm[(size_t)slot * N + j];
    for (int i = lane; i < d; i += 32) {
      const double2 g = sG[i * BT + c];
      const auto ph = sP[i * BT + c];
      gout[(size_t)j * d + i] =
          make_double2((g.x - (double)ph.x * rad) * inv_r, (g.y - (double)ph.y * rad) * inv_r);
    }
  }
}

// columns per CTA of the final pass: as many as fit 96 KiB of staging
template <typename T> int finish_cols(int d) {
  int cw = 32;
  while (cw > 8 && (size_t)d * cw * (sizeof(double2) + 2 * sizeof(T)) > 96 * 1024) cw >>= 1;
  return cw;
}

template <typename T> size_t lse_smem(int d, int R) {
  const size_t BT = 16 * (size_t)R;
  return (8 * (size_t)d * BT + 2 * BT * (BT + 4)) * sizeof(T);
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
  const size_t smem_tile = lse_smem<T>(a.d, R);
  const long long items = (long long)a.count * a.ntiles;
  int grid = 0;
  cudaError_t e;
  // s: the search's tile pass over the planes
  GramSource src{};
  src.perturb = true;       // candidates given as planes: no generation
  src.planes = a.planes;
  if constexpr (sizeof(T) == 4)
    e = launch_gram_f32(a.N, a.d, a.count, src, a.smax, nullptr, num_sms, s);
  else
    e = launch_gram_f64(a.N, a.d, a.count, src, a.smax, num_sms, s);
  if (e != cudaSuccess) return e;
  if ((e = lse_grid(k_lse_tile<T, R>, smem_tile, items, num_sms, &grid)) != cudaSuccess) return e;
  k_lse_tile<T, R><<<grid, kLseThreads, smem_tile, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_lse_total<T><<<a.count, kLseThreads, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.grad) {
    constexpr int BT = 16 * R;
    const size_t block_smem = (size_t)a.d * BT * (sizeof(double2) + 2 * sizeof(T));
    if (block_smem <= 96 * 1024) {
      k_lse_finish_block<T, R><<<(unsigned)((long long)a.count * a.nb), kLseThreads, block_smem,
                                 s>>>(a);
    } else {
      const int cw = finish_cols<T>(a.d);
      const long long ctas = (long long)a.count * ((a.N + cw - 1) / cw);
      const size_t smem = (size_t)a.d * cw * (sizeof(double2) + 2 * sizeof(T));
      k_lse_finish<T, R><<<(unsigned)ctas, kLseThreads, smem, s>>>(a, cw);
    }
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
cudaError_t lse_run(int N, int d, int count, const double* v, double delta,
                    const double* deltas, void* scratch,
                    double* out, double* grad, int num_sms, cudaStream_t s) {
  const LseLayout<T> L = lse_layout<T>(N, d, count);
  unsigned char* b = static_cast<unsigned char*>(scratch);
  LseArgs<T> a;
  a.N = N; a.d = d; a.nb = L.nb; a.ntiles = L.ntiles; a.count = count;
  a.delta = delta;
  a.deltas = deltas;
  a.v = v;
  a.planes = reinterpret_cast<T*>(b + L.o_planes);
  a.rnorm = reinterpret_cast<T*>(b + L.o_rnorm);
  a.bad = reinterpret_cast<uint32_t*>(b + L.o_bad);
  a.vec = (N % (16 / (int)sizeof(T)) == 0) ? 1 : 0;
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
  return f64 ? lse_run<double>(N, d, count, v, delta, nullptr, scratch, out, grad, num_sms, s)
             : lse_run<float>(N, d, count, v, delta, nullptr, scratch, out, grad, num_sms, s);
}

cudaError_t launch_lse_deltas(int N, int d, int count, const double* v, const double* deltas,
                              bool f64, void* scratch, double* out, double* grad, int num_sms,
                              cudaStream_t s) {
  if (N < 2 || d < 1 || d > kMaxD || count < 1 || !deltas) return cudaErrorInvalidValue;
  return f64 ? lse_run<double>(N, d, count, v, 0.0, deltas, scratch, out, grad, num_sms, s)
             : lse_run<float>(N, d, count, v, 0.0, deltas, scratch, out, grad, num_sms, s);
}

cudaError_t init_lse_attributes(int optin) {
  cudaError_t e;
  if ((e = lse_allow(k_lse_tile<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<double, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_tile<double, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish<double, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish_block<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish_block<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish_block<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish_block<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish_block<double, 2>, optin)) != cudaSuccess) return e;
  if ((e = lse_allow(k_lse_finish_block<double, 1>, optin)) != cudaSuccess) return e;
  return lse_allow(k_lse_finish<double, 1>, optin);
}

}  // namespace trstmi
