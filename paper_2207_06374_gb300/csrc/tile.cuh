// Device helpers shared by the SIMT tile kernels (the search's Gram passes
// and the smooth-maximum objective): pair rounding, tile enumeration, block
// reductions and the R x R complex micro-tile of the upper-triangle Gram.
#pragma once

#include "kernels.h"

namespace trstmi {

// |G_jk|^2 from its accumulated parts, rounded explicitly so that every
// kernel that scores a pair gives the same bits (the accumulation itself is
// the sequential chain over i of MicroTile::step).
__device__ __forceinline__ float pair_abs2(float re, float im) {
  return __fmaf_rn(re, re, __fmul_rn(im, im));
}
__device__ __forceinline__ double pair_abs2(double re, double im) {
  return __fma_rn(re, re, __dmul_rn(im, im));
}

// Upper-triangle tile tau (column-major over tiles with I <= J) -> (I, J).
__device__ __forceinline__ void tile_coords(int tau, int& I, int& J) {
  int j = (int)((sqrtf(8.0f * (float)tau + 1.0f) - 1.0f) * 0.5f);
  while ((j + 1) * (j + 2) / 2 <= tau) ++j;
  while (j * (j + 1) / 2 > tau) --j;
  J = j;
  I = tau - j * (j + 1) / 2;
}

template <typename T> __device__ __forceinline__ T block_max(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

// R consecutive shared-memory values (R * sizeof(T)-aligned) in vector loads.
template <typename T, int R>
__device__ __forceinline__ void load_run(const T* p, T (&v)[R]) {
  if constexpr (sizeof(T) == 4 && R == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (sizeof(T) == 4 && R == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else if constexpr (sizeof(T) == 8 && R >= 2) {
#pragma unroll
    for (int h = 0; h < R; h += 2) {
      const double2 q = *reinterpret_cast<const double2*>(p + h);
      v[h] = q.x; v[h + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int x = 0; x < R; ++x) v[x] = p[x];
  }
}

// R x R complex accumulators of a micro-tile and one step i of their chains:
//   Re += a_ij a_ik + b_ij b_ik,  Im += a_ij b_ik - b_ij a_ik,
// each as two fused multiply-adds in that order, so every pair's value is a
// fixed sequence of roundings whatever the micro-tile shape.
template <typename T, int R, bool Packed = (sizeof(T) == 4 && R % 2 == 0)>
struct MicroTile {
  T re[R][R], im[R][R];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) { re[x][y] = T(0); im[x][y] = T(0); }
  }
  __device__ __forceinline__ void step(const T (&ar)[R], const T (&ai)[R], const T (&br)[R],
                                       const T (&bi)[R]) {
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) {
        re[x][y] = fma(ar[x], br[y], fma(ai[x], bi[y], re[x][y]));
        im[x][y] = fma(ar[x], bi[y], fma(-ai[x], br[y], im[x][y]));
      }
  }
  __device__ __forceinline__ T get_re(int x, int y) const { return re[x][y]; }
  __device__ __forceinline__ T get_im(int x, int y) const { return im[x][y]; }
};

// binary32 with an even R: neighbouring columns y, y+1 in one packed pair,
// updated by paired fused multiply-adds (each lane rounds exactly as the
// scalar fma, so the values are the same bits) in half the instructions
template <int R>
struct MicroTile<float, R, true> {
  float2 re[R][R / 2], im[R][R / 2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int h = 0; h < R / 2; ++h) { re[x][h] = make_float2(0.f, 0.f); im[x][h] = re[x][h]; }
  }
  __device__ __forceinline__ void step(const float (&ar)[R], const float (&ai)[R],
                                       const float (&br)[R], const float (&bi)[R]) {
#pragma unroll
    for (int x = 0; x < R; ++x) {
      const float2 a = make_float2(ar[x], ar[x]);
      const float2 b = make_float2(ai[x], ai[x]);
      const float2 nb = make_float2(-ai[x], -ai[x]);
#pragma unroll
      for (int h = 0; h < R / 2; ++h) {
        const float2 r = make_float2(br[2 * h], br[2 * h + 1]);
        const float2 q = make_float2(bi[2 * h], bi[2 * h + 1]);
        re[x][h] = __ffma2_rn(a, r, __ffma2_rn(b, q, re[x][h]));
        im[x][h] = __ffma2_rn(a, q, __ffma2_rn(nb, r, im[x][h]));
      }
    }
  }
  __device__ __forceinline__ float get_re(int x, int y) const {
    return (y & 1) ? re[x][y >> 1].y : re[x][y >> 1].x;
  }
  __device__ __forceinline__ float get_im(int x, int y) const {
    return (y & 1) ? im[x][y >> 1].y : im[x][y >> 1].x;
  }
};

// The reduction of tile (I, J) of width BT = 16 R once its column blocks are
// in shared memory: sI holds block I as [i][column] planes (d x BT real
// parts, then d x BT imaginary parts) and sJ block J in the same layout
// (sJ == sI on a diagonal tile).  Thread (ty, tx) of the 16 x 16 CTA owns
// rows R ty .. R ty + R-1 and columns R tx .. R tx + R-1 of the tile and
// reads R consecutive values per plane in one vector load each.  Returns the
// thread's max of |G_jk|^2 over its pairs j < k < N and appends the pairs at
// or above thr when filter != nullptr.
template <typename T, int R>
__device__ __forceinline__ T tile_pairs_max(const T* sIre, const T* sIim, const T* sJ, int d,
                                            int N, int I, int J, T thr,
                                            const PairFilter* filter) {
  constexpr int BT = 16 * R;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const T* bRe = sJ;
  const T* bIm = sJ + (size_t)d * BT;
  MicroTile<T, R> acc;
  acc.zero();
#pragma unroll 2
  for (int i = 0; i < d; ++i) {
    T ar[R], ai[R], br[R], bi[R];
    load_run<T, R>(sIre + i * BT + R * ty, ar);
    load_run<T, R>(sIim + i * BT + R * ty, ai);
    load_run<T, R>(bRe + i * BT + R * tx, br);
    load_run<T, R>(bIm + i * BT + R * tx, bi);
    acc.step(ar, ai, br, bi);
  }
  T m = T(0);
  if (filter && filter->local) {
    // the threshold from this tile's own maximum (see PairFilter::local)
    __shared__ T red[8];
    __shared__ T tile_max;
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) {
        const int gj = I * BT + R * ty + x, gk = J * BT + R * tx + y;
        if (gj < gk && gk < N) m = fmax(m, pair_abs2(acc.get_re(x, y), acc.get_im(x, y)));
      }
    const T bm = block_max<T>(m, red);
    if (threadIdx.x == 0) tile_max = bm;
    __syncthreads();
    const float lo = fmaxf(sqrtf((float)tile_max) - filter->margin, 0.0f);
    thr = (T)(lo * lo);
  }
#pragma unroll
  for (int x = 0; x < R; ++x)
#pragma unroll
    for (int y = 0; y < R; ++y) {
      const int gj = I * BT + R * ty + x, gk = J * BT + R * tx + y;
      const T v = pair_abs2(acc.get_re(x, y), acc.get_im(x, y));
      if (gj < gk && gk < N) {
        m = fmax(m, v);
        if (filter && v >= thr) {
          const uint32_t idx = atomicAdd(filter->npairs, 1u);
          if (idx < filter->cap) filter->pairs[idx] = make_uint2((unsigned)gj, (unsigned)gk);
          else atomicExch(filter->overflow, 1u);
        }
      }
    }
  return m;
}

// ------------------------------------------- asynchronous tile copies
__device__ __forceinline__ uint32_t shared_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// B = 4, 8 or 16 bytes from global to shared memory, zeros when !valid (src
// must be a valid address either way); both addresses B-byte aligned
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  if constexpr (B == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(shared_addr(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(shared_addr(dst)),
                 "l"(src), "n"(B), "r"(valid ? B : 0)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int Pending> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(Pending) : "memory");
}

// Issues the copies of column blocks I and J (J only off the diagonal) of a
// frame held as planes (pre: d x N real parts, then d x N imaginary parts)
// into dst: block I as d x BT real, d x BT imaginary, then block J; columns
// past N are zeros.  vec: N a multiple of 16 / sizeof(T) and pre 16-byte
// aligned, so every run of 16 bytes is one aligned copy.
template <typename T, int BT>
__device__ __forceinline__ void prefetch_blocks(const T* pre, int d, int N, int I, int J, T* dst,
                                                bool vec) {
  constexpr int V = 16 / (int)sizeof(T);
  const T* pim = pre + (size_t)d * N;
  for (int blk = 0; blk < (I == J ? 1 : 2); ++blk) {
    const int c0 = (blk == 0 ? I : J) * BT;
    T* ore = dst + (size_t)blk * 2 * d * BT;
    T* oim = ore + (size_t)d * BT;
    if (vec) {
      for (int q = threadIdx.x; q < d * (BT / V); q += blockDim.x) {
        const int i = q / (BT / V), cv = q % (BT / V);
        const int gj = c0 + V * cv;
        const bool ok = gj < N;
        const size_t g = ok ? (size_t)i * N + gj : 0;
        cp_async<16>(ore + i * BT + V * cv, pre + g, ok);
        cp_async<16>(oim + i * BT + V * cv, pim + g, ok);
      }
    } else {
      for (int q = threadIdx.x; q < d * BT; q += blockDim.x) {
        const int i = q / BT, loc = q % BT;
        const int gj = c0 + loc;
        const bool ok = gj < N;
        const size_t g = ok ? (size_t)i * N + gj : 0;
        cp_async<(int)sizeof(T)>(ore + q, pre + g, ok);
        cp_async<(int)sizeof(T)>(oim + q, pim + g, ok);
      }
    }
  }
}

}  // namespace trstmi
