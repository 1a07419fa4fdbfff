// SIMT kernels of the TRSTMI search: candidate generation, the tiled
// upper-triangle Gram with a fused |G|^2 / max epilogue (binary32 and
// binary64), and the per-iteration select / accept / commit kernels.
//
// Method (arXiv 2207.06374): coherence mu(Phi) = max_{j != k} |<phi_j, phi_k>|
// (Sec. "Introduction"); only the upper triangle j < k is formed (Sec.
// "Optimization procedure"); columns are renormalised after every
// perturbation so the search is unconstrained (Remark on normalisation).
#include <algorithm>

#include "kernels.h"
#include "philox.cuh"
#include "tile.cuh"

namespace trstmi {

// ----------------------------------------------------- rounding helpers
// Generation uses explicitly rounded operations so that the same candidate
// is bit-identical wherever it is regenerated (scoring, commit, copies).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

template <typename T> __device__ __forceinline__ void cn_draw(uint32_t ua, uint32_t ub, T& re, T& im);
template <> __device__ __forceinline__ void cn_draw<float>(uint32_t ua, uint32_t ub, float& re, float& im) {
  cn_from_u32_f32(ua, ub, re, im);
}
template <> __device__ __forceinline__ void cn_draw<double>(uint32_t ua, uint32_t ub, double& re, double& im) {
  cn_from_u32_f64(ua, ub, re, im);
}

// Column j of normalise(Phi + delta * Z_{t,c}) (tag 0), or of the initial
// draw normalise(Z_init) (tag 1, phi == nullptr), written to
// out_re[i*stride], out_im[i*stride].  Returns false for a zero column.
// Entry i of phi is read before out[i] is written and never again, so the
// output may alias the input column (in-place commit).
template <typename T>
__device__ bool gen_column(const typename Cplx<T>::type* phi, int d, int j,
                           uint64_t seed, uint32_t c, uint32_t t, uint32_t tag, T delta,
                           T* out_re, T* out_im, int stride) {
  const uint32_t k0 = seed_lo(seed), k1 = seed_hi(seed);
  const int P = (d + 1) >> 1;
  const typename Cplx<T>::type* col = phi ? phi + (size_t)j * d : nullptr;
  T s = T(0);
  for (int p = 0; p < P; ++p) {
    const PhiloxOut u = philox4x32_10((uint32_t)j * (uint32_t)P + (uint32_t)p, c, t, tag, k0, k1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * p + h;
      if (i < d) {
        T zr, zi;
        cn_draw<T>(u.x[2 * h], u.x[2 * h + 1], zr, zi);
        T xr = zr, xi = zi;
        if (col) {
          const auto v = col[i];
          xr = add_rn(v.x, mul_rn(delta, zr));
          xi = add_rn(v.y, mul_rn(delta, zi));
        }
        out_re[i * stride] = xr;
        out_im[i * stride] = xi;
        s = add_rn(s, add_rn(mul_rn(xr, xr), mul_rn(xi, xi)));
      }
    }
  }
  if (!(s > T(0))) {
    for (int i = 0; i < d; ++i) { out_re[i * stride] = T(0); out_im[i * stride] = T(0); }
    return false;
  }
  const T nrm = sqrt_rn(s);
  for (int i = 0; i < d; ++i) {
    out_re[i * stride] = div_rn(out_re[i * stride], nrm);
    out_im[i * stride] = div_rn(out_im[i * stride], nrm);
  }
  return true;
}

// CTA-cooperative form of gen_column for all N columns of candidate (c, t)
// into [i][column] planes of row pitch `stride`: the draws (Philox,
// Box-Muller, phi + delta z) are spread over the (column, entry pair) items,
// then one thread per column forms the squared norm in the same sequential
// order over i and divides, so every value has the bits gen_column gives it.
// Returns (in every thread) whether a column had zero norm.  Begins and ends
// with a CTA barrier.
template <typename T>
__device__ bool gen_candidate_cta(const typename Cplx<T>::type* phi, int N, int d, uint64_t seed,
                                  uint32_t c, uint32_t t, T delta, T* out_re, T* out_im,
                                  int stride, int* zero_flag) {
  const uint32_t k0 = seed_lo(seed), k1 = seed_hi(seed);
  const int P = (d + 1) >> 1;
  __syncthreads();
  for (int q = threadIdx.x; q < N * P; q += blockDim.x) {
    // consecutive threads take consecutive columns of one entry pair, so their
    // shared-memory stores fall in consecutive words
    const int p = q / N, j = q - p * N;
    const PhiloxOut u = philox4x32_10((uint32_t)j * (uint32_t)P + (uint32_t)p, c, t, 0u, k0, k1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * p + h;
      if (i < d) {
        T zr, zi;
        cn_draw<T>(u.x[2 * h], u.x[2 * h + 1], zr, zi);
        const auto v = phi[(size_t)j * d + i];
        out_re[i * stride + j] = add_rn(v.x, mul_rn(delta, zr));
        out_im[i * stride + j] = add_rn(v.y, mul_rn(delta, zi));
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    T s = T(0);
    for (int i = 0; i < d; ++i) {
      const T xr = out_re[i * stride + j], xi = out_im[i * stride + j];
      s = add_rn(s, add_rn(mul_rn(xr, xr), mul_rn(xi, xi)));
    }
    if (!(s > T(0))) {
      for (int i = 0; i < d; ++i) { out_re[i * stride + j] = T(0); out_im[i * stride + j] = T(0); }
      *zero_flag = 1;
      continue;
    }
    const T nrm = sqrt_rn(s);
    for (int i = 0; i < d; ++i) {
      out_re[i * stride + j] = div_rn(out_re[i * stride + j], nrm);
      out_im[i * stride + j] = div_rn(out_im[i * stride + j], nrm);
    }
  }
  __syncthreads();
  return *zero_flag != 0;
}

// Warp-cooperative form of gen_column for an interleaved column in global
// memory: lane l draws the entry pairs p = l, l + 32, ...; the squared norm
// is reduced across the warp.  All 32 lanes must call it.
template <typename T>
__device__ bool gen_column_warp(const typename Cplx<T>::type* phi, int d, int j, uint64_t seed,
                                uint32_t c, uint32_t t, uint32_t tag, T delta,
                                typename Cplx<T>::type* out, int lane) {
  const uint32_t k0 = seed_lo(seed), k1 = seed_hi(seed);
  const int P = (d + 1) >> 1;
  const typename Cplx<T>::type* col = phi ? phi + (size_t)j * d : nullptr;
  typename Cplx<T>::type* o = out + (size_t)j * d;
  // one entry per lane (the two lanes of an entry pair both run its Philox
  // call), so every lane carries a Box-Muller transform
  T s = T(0);
  for (int i = lane; i < d; i += 32) {
    const int p = i >> 1, h = i & 1;
    const PhiloxOut u = philox4x32_10((uint32_t)j * (uint32_t)P + (uint32_t)p, c, t, tag, k0, k1);
    T zr, zi;
    cn_draw<T>(u.x[2 * h], u.x[2 * h + 1], zr, zi);
    T xr = zr, xi = zi;
    if (col) {
      const auto v = col[i];
      xr = add_rn(v.x, mul_rn(delta, zr));
      xi = add_rn(v.y, mul_rn(delta, zi));
    }
    o[i].x = xr;
    o[i].y = xi;
    s = add_rn(s, add_rn(mul_rn(xr, xr), mul_rn(xi, xi)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (!(s > T(0))) return false;
  const T nrm = sqrt_rn(s);
  for (int i = lane; i < d; i += 32) { o[i].x = div_rn(o[i].x, nrm); o[i].y = div_rn(o[i].y, nrm); }
  return true;
}

// Column j of a stored frame, optionally renormalised.
template <typename T>
__device__ bool load_column(const typename Cplx<T>::type* __restrict__ frame, int d, int j,
                            bool normalize, T* out_re, T* out_im, int stride) {
  const typename Cplx<T>::type* col = frame + (size_t)j * d;
  T s = T(0);
  for (int i = 0; i < d; ++i) {
    const auto v = col[i];
    out_re[i * stride] = v.x;
    out_im[i * stride] = v.y;
    s = add_rn(s, add_rn(mul_rn(v.x, v.x), mul_rn(v.y, v.y)));
  }
  if (!normalize) return true;
  if (!(s > T(0))) return false;
  const T nrm = sqrt_rn(s);
  for (int i = 0; i < d; ++i) {
    out_re[i * stride] = div_rn(out_re[i * stride], nrm);
    out_im[i * stride] = div_rn(out_im[i * stride], nrm);
  }
  return true;
}

template <typename T> struct GramArgs {
  int N, d, nb, ntiles, nslots;
  GramSource src;
  typename Mu2Bits<T>::type* out;
  PairFilter filter;
  bool has_filter;
};

// One work item of a Gram pass: tile (I <= J) of one frame, either the
// candidate normalise(Phi + delta Z_{t,c}) or a stored frame.
struct TileItem {
  int N, d, I, J;
  bool perturb, normalize;
  const void* phi;   // float2* / double2*: base frame (perturb) or the frame itself
  uint64_t seed;
  uint32_t c, t;
  double delta;
  const void* planes = nullptr;   // candidate drawn already: [i][column] re, then im planes
};

// The CTA (256 threads, 16 x 16) scores tile (I, J) of width BT = 16 R.
// Column blocks I and J are generated (or loaded) into shared memory as
// [i][column] planes of real and imaginary parts; each thread accumulates an
// R x R micro-tile of
//   Re G_jk = sum_i a_ij a_ik + b_ij b_ik,  Im G_jk = sum_i a_ij b_ik - b_ij a_ik
// as a sequential chain over i (tile_pairs_max), so a pair's |G_jk|^2 does
// not depend on the tile shape.  Returns this thread's max over its pairs
// j < k < N (and appends the pairs at or above thr when filter != nullptr).
// Begins with a CTA barrier; *zero_col is set if a column had zero norm.
template <typename T, int R>
__device__ T score_tile(const TileItem& it, T* sm, int* zero_col, T thr,
                        const PairFilter* filter) {
  constexpr int BT = 16 * R;
  using C = typename Cplx<T>::type;
  const int d = it.d, N = it.N, I = it.I, J = it.J;
  T* sIre = sm;
  T* sIim = sm + (size_t)d * BT;
  T* sJre = sm + (size_t)2 * d * BT;
  T* sJim = sm + (size_t)3 * d * BT;
  const bool diag = (I == J);
  __syncthreads();
  const int ncols = diag ? BT : 2 * BT;
  if (it.planes) {
    // coalesced copy of the two column blocks out of the drawn candidate
    // (BT is a compile-time power of two: the index split is shifts)
    const T* pre = reinterpret_cast<const T*>(it.planes);
    const T* pim = pre + (size_t)d * N;
    for (int blk = 0; blk < (diag ? 1 : 2); ++blk) {
      const int c0 = (blk == 0 ? I : J) * BT;
      T* ore = blk == 0 ? sIre : sJre;
      T* oim = blk == 0 ? sIim : sJim;
      for (int q = threadIdx.x; q < d * BT; q += blockDim.x) {
        const int i = q / BT, loc = q % BT;
        const int gj = c0 + loc;
        const size_t g = (size_t)i * N + gj;
        ore[q] = gj < N ? pre[g] : T(0);
        oim[q] = gj < N ? pim[g] : T(0);
      }
    }
  } else
  for (int q = threadIdx.x; q < ncols; q += blockDim.x) {
    const int blk = q / BT, loc = q - blk * BT;
    const int gj = (blk == 0 ? I : J) * BT + loc;
    T* ore = (blk == 0 ? sIre : sJre) + loc;
    T* oim = (blk == 0 ? sIim : sJim) + loc;
    bool ok = true;
    if (gj < N) {
      if (it.perturb)
        ok = gen_column<T>(reinterpret_cast<const C*>(it.phi), d, gj, it.seed, it.c, it.t, 0u,
                           (T)it.delta, ore, oim, BT);
      else
        ok = load_column<T>(reinterpret_cast<const C*>(it.phi), d, gj, it.normalize, ore, oim, BT);
    } else {
      for (int i = 0; i < d; ++i) { ore[i * BT] = T(0); oim[i * BT] = T(0); }
    }
    if (!ok) *zero_col = 1;
  }
  __syncthreads();
  return tile_pairs_max<T, R>(sIre, sIim, diag ? sIre : sJre, d, N, I, J, thr, filter);
}

// Gram pass over nslots frames (candidates of one instance, or stored
// frames), one CTA per (slot, tile) work item, grid-stride.
// binary32: at most 85 registers, so three 256-thread CTAs per SM hide the
// loads of one CTA's next tile behind the others' arithmetic; binary64 keeps
// its larger micro-tile in registers
template <typename T> struct TileCtas { static constexpr int value = sizeof(T) == 4 ? 3 : 1; };

template <typename T, int R>
__global__ void __launch_bounds__(256, TileCtas<T>::value) k_gram_tile(const GramArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[8];
  __shared__ int zero_col;
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int d = a.d, N = a.N;

  const GramSource& src = a.src;
  if (src.gate && *src.gate == 0u) return;
  uint32_t t = src.t;
  T delta = (T)src.delta;
  if (src.st) {
    if (!src.st->active) return;
    t = src.st->t + 1u;
    delta = (T)src.st->delta_used;
  }
  T thr = T(-1);
  if (a.has_filter && !a.filter.local) {
    const float lo = filter_lo(a.filter);
    thr = (T)(lo * lo);
  }
  const long long nitems = (long long)a.nslots * a.ntiles;
  for (long long w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int slot = (int)(w / a.ntiles);
    const int tau = (int)(w - (long long)slot * a.ntiles);
    TileItem it;
    it.N = N; it.d = d;
    tile_coords(tau, it.I, it.J);
    it.perturb = src.perturb;
    it.normalize = src.normalize;
    it.seed = src.seed;
    it.t = t;
    it.delta = (double)delta;
    if (src.perturb) {
      it.phi = src.phi;
      it.c = src.cand_list ? src.cand_list[slot] : src.c0 + (uint32_t)slot;
      if (src.planes)
        it.planes = reinterpret_cast<const T*>(src.planes) + (size_t)slot * 2 * d * N;
    } else {
      it.phi = reinterpret_cast<const typename Cplx<T>::type*>(src.phi) + (size_t)slot * d * N;
      it.c = 0u;
    }
    if (threadIdx.x == 0) zero_col = 0;
    T m = score_tile<T, R>(it, sm, &zero_col, thr, a.has_filter ? &a.filter : nullptr);
    if (zero_col && src.st && threadIdx.x == 0)
      atomicOr(&const_cast<DevState*>(src.st)->error, (uint32_t)kErrZeroColumn);
    m = block_max<T>(m, red);
    if (threadIdx.x == 0) atomic_max_nonneg(a.out + slot, m);
    __syncthreads();
  }
}

// ------------------------------------------- binary32 pass over drawn planes
// The tile pass when the iteration's candidates are already drawn (planes,
// [i][column] real then imaginary, 2 d N floats per candidate): the column
// blocks of the CTA's next work item are copied into a second shared-memory
// stage with asynchronous copies while the current item is reduced, so the
// copy latency hides behind the arithmetic of the same CTA.  The reduction is
// tile_pairs_max, the scores the same bits as k_gram_tile's.

// Issues the copies of work item w's column blocks into stage dst (block I,
// then block J unless the tile is diagonal; each d x BT real, d x BT
// imaginary).  vec: N % 4 == 0 and a 16-byte aligned planes array, so every
// run of 4 columns is one aligned 16-byte copy.
template <int R>
__device__ __forceinline__ void prefetch_planes(const GramArgs<float>& a, long long w, float* dst,
                                                bool vec) {
  const int slot = (int)(w / a.ntiles);
  int I, J;
  tile_coords((int)(w - (long long)slot * a.ntiles), I, J);
  const float* pre = reinterpret_cast<const float*>(a.src.planes) + (size_t)slot * 2 * a.d * a.N;
  prefetch_blocks<float, 16 * R>(pre, a.d, a.N, I, J, dst, vec);
}

template <int R>
__global__ void __launch_bounds__(256, 3) k_gram_planes(const GramArgs<float> a, int vec) {
  constexpr int BT = 16 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float red[8];
  float* const stage0 = reinterpret_cast<float*>(smem_raw);
  const size_t stage_floats = (size_t)4 * a.d * BT;
  const GramSource& src = a.src;
  if (src.gate && *src.gate == 0u) return;
  if (src.st && !src.st->active) return;
  float thr = -1.f;
  if (a.has_filter && !a.filter.local) {
    const float lo = filter_lo(a.filter);
    thr = lo * lo;
  }
  const long long nitems = (long long)a.nslots * a.ntiles;
  long long w = blockIdx.x;
  if (w < nitems) prefetch_planes<R>(a, w, stage0, vec != 0);
  cp_async_commit();
  for (int sg = 0; w < nitems; w += gridDim.x, sg ^= 1) {
    const long long wn = w + gridDim.x;
    if (wn < nitems) prefetch_planes<R>(a, wn, stage0 + (sg ^ 1) * stage_floats, vec != 0);
    cp_async_commit();
    cp_async_wait<1>();   // this thread's copies of item w have landed ...
    __syncthreads();      // ... and every other thread's
    const int slot = (int)(w / a.ntiles);
    int I, J;
    tile_coords((int)(w - (long long)slot * a.ntiles), I, J);
    const float* sI = stage0 + sg * stage_floats;
    const float* sJ = I == J ? sI : sI + (size_t)2 * a.d * BT;
    float m = tile_pairs_max<float, R>(sI, sI + (size_t)a.d * BT, sJ, a.d, a.N, I, J, thr,
                                       a.has_filter ? &a.filter : nullptr);
    m = block_max<float>(m, red);
    if (threadIdx.x == 0) atomic_max_nonneg(a.out + slot, m);
    __syncthreads();      // stage sg is free for the copies issued next round
  }
  cp_async_wait<0>();
}

// Candidates drawn once for the tile pass.  Many columns (the K candidates of
// an iteration): k_gen_planes_f32, one thread per column running gen_column.
// Few columns (the top-k survivors), where that leaves most SMs idle:
// k_draw_planes_tiled_f32 (below) spreads the draws over (column, entry pair)
// items and gives every value the bits gen_column gives it.
struct PlanesDraw {
  int N, d, P, count;
  const float2* phi;
  uint64_t seed;
  uint32_t c0, t;
  float delta;
  float* planes;
  const uint32_t* cand_list;
  const uint32_t* gate;
  DevState* st;
};

__device__ __forceinline__ bool planes_draw_setup(PlanesDraw& a) {
  if (a.gate && *a.gate == 0u) return false;
  if (a.st) {
    if (!a.st->active) return false;
    a.t = a.st->t + 1u;
    a.delta = (float)a.st->delta_used;
  }
  return true;
}

__global__ void k_gen_planes_f32(PlanesDraw a) {
  if (!planes_draw_setup(a)) return;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (long long)a.count * a.N) return;
  const int slot = (int)(g / a.N), j = (int)(g - (long long)slot * a.N);
  float* pre = a.planes + (size_t)slot * 2 * a.d * a.N;
  float* pim = pre + (size_t)a.d * a.N;
  const uint32_t c = a.cand_list ? a.cand_list[slot] : a.c0 + (uint32_t)slot;
  if (!gen_column<float>(a.phi, a.d, j, a.seed, c, a.t, 0u, a.delta, pre + j, pim + j, a.N) && a.st)
    atomicOr(&a.st->error, (uint32_t)kErrZeroColumn);
}

// Few columns, one pass: a CTA takes 32 consecutive columns of one slot.  Its
// threads draw the (column, entry pair) items (Philox, Box-Muller, phi +
// delta z) into shared memory as [part][i][column]; thread t < 32 then forms
// column t's squared norm in gen_column's order (i ascending) and all threads
// write the divided entries to the planes, 32 consecutive columns per row, so
// the stores are coalesced.  Every value has the bits gen_column gives it.
constexpr int kDrawCols = 32;
__global__ void __launch_bounds__(256) k_draw_planes_tiled_f32(PlanesDraw a) {
  extern __shared__ __align__(16) float xs[];   // [2][d][kDrawCols]
  __shared__ float nrm[kDrawCols];
  __shared__ int bad[kDrawCols];
  if (!planes_draw_setup(a)) return;
  const int d = a.d, N = a.N, P = a.P;
  const int tiles = (N + kDrawCols - 1) / kDrawCols;
  const int slot = blockIdx.x / tiles, c0 = (blockIdx.x - slot * tiles) * kDrawCols;
  const uint32_t c = a.cand_list ? a.cand_list[slot] : a.c0 + (uint32_t)slot;
  float* xre = xs;
  float* xim = xs + (size_t)d * kDrawCols;
  for (int q = threadIdx.x; q < kDrawCols * P; q += blockDim.x) {
    const int cl = q % kDrawCols, p = q / kDrawCols, j = c0 + cl;
    if (j >= N) continue;
    const PhiloxOut u = philox4x32_10((uint32_t)j * (uint32_t)P + (uint32_t)p, c, a.t, 0u,
                                      seed_lo(a.seed), seed_hi(a.seed));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * p + h;
      if (i < d) {
        float zr, zi;
        cn_draw<float>(u.x[2 * h], u.x[2 * h + 1], zr, zi);
        const float2 v = a.phi[(size_t)j * d + i];
        xre[i * kDrawCols + cl] = add_rn(v.x, mul_rn(a.delta, zr));
        xim[i * kDrawCols + cl] = add_rn(v.y, mul_rn(a.delta, zi));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < kDrawCols) {
    const int cl = threadIdx.x;
    float sq = 0.f;
    if (c0 + cl < N)
      for (int i = 0; i < d; ++i) {
        const float xr = xre[i * kDrawCols + cl], xi = xim[i * kDrawCols + cl];
        sq = add_rn(sq, add_rn(mul_rn(xr, xr), mul_rn(xi, xi)));
      }
    bad[cl] = (c0 + cl < N) && !(sq > 0.f);
    nrm[cl] = sq > 0.f ? sqrt_rn(sq) : 0.f;
    if (bad[cl] && a.st) atomicOr(&a.st->error, (uint32_t)kErrZeroColumn);
  }
  __syncthreads();
  float* pre = a.planes + (size_t)slot * 2 * d * N;
  float* pim = pre + (size_t)d * N;
  for (int q = threadIdx.x; q < d * kDrawCols; q += blockDim.x) {
    const int cl = q % kDrawCols, i = q / kDrawCols, j = c0 + cl;
    if (j >= N) continue;
    const bool z = bad[cl] != 0;
    pre[(size_t)i * N + j] = z ? 0.f : div_rn(xre[q], nrm[cl]);
    pim[(size_t)i * N + j] = z ? 0.f : div_rn(xim[q], nrm[cl]);
  }
}

cudaError_t launch_gen_planes_f32(int N, int d, int count, const float2* phi, uint64_t seed,
                                  uint32_t c0, DevState* st, uint32_t t, double delta,
                                  float* planes, cudaStream_t s, const uint32_t* cand_list,
                                  const uint32_t* gate) {
  if (count < 1) return cudaSuccess;
  PlanesDraw a{N, d, (d + 1) / 2, count, phi, seed, c0, t, (float)delta, planes, cand_list, gate,
               st};
  const long long cols = (long long)count * N;
  if (cols >= 65536) {
    k_gen_planes_f32<<<(unsigned)((cols + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  const long long tiles = (long long)count * ((N + kDrawCols - 1) / kDrawCols);
  const size_t smem = (size_t)2 * d * kDrawCols * sizeof(float);
  k_draw_planes_tiled_f32<<<(unsigned)tiles, 256, smem, s>>>(a);
  return cudaGetLastError();
}

// shared memory of the double-buffered binary32 pass (two stages)
constexpr size_t kPlanesSmemMax = 200 * 1024;

template <typename T> static size_t gram_smem(int d, int R) {
  return (size_t)4 * d * 16 * R * sizeof(T);
}

template <typename T> static int pick_R(int N, int d) {
  int R = 4;
  while (R > 1 && 16 * R >= 2 * N) R >>= 1;          // do not pad tiny N
  while (R > 1 && gram_smem<T>(d, R) > 200 * 1024) R >>= 1;
  return R;
}

template <typename T>
static cudaError_t launch_gram(int N, int d, int nslots, const GramSource& src,
                               typename Mu2Bits<T>::type* out, const PairFilter* filter,
                               int num_sms, cudaStream_t s) {
  if (N < 1 || d < 1 || d > kMaxD || nslots < 0) return cudaErrorInvalidValue;
  if (nslots == 0) return cudaSuccess;
  const int R = pick_R<T>(N, d);
  const int BT = 16 * R;
  GramArgs<T> a;
  a.N = N; a.d = d; a.nb = (N + BT - 1) / BT; a.ntiles = a.nb * (a.nb + 1) / 2;
  a.nslots = nslots; a.src = src; a.out = out;
  a.has_filter = filter != nullptr;
  if (filter) a.filter = *filter; else a.filter = PairFilter{};
  const size_t smem = gram_smem<T>(d, R);
  const long long items = (long long)nslots * a.ntiles;
  int per_sm = 1;
  if constexpr (sizeof(T) == 4) {
    // candidates already drawn: the double-buffered pass when two stages fit
    if (src.planes && 2 * smem <= kPlanesSmemMax) {
      const int vec = (N % 4 == 0 && reinterpret_cast<uintptr_t>(src.planes) % 16 == 0) ? 1 : 0;
      cudaError_t oe = R == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_planes<4>, 256, 2 * smem)
                     : R == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_planes<2>, 256, 2 * smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_planes<1>, 256, 2 * smem);
      if (oe != cudaSuccess) return oe;
      per_sm = std::max(per_sm, 1);
      const int grid = (int)std::min<long long>(items, (long long)num_sms * per_sm);
      switch (R) {
        case 4: k_gram_planes<4><<<grid, 256, 2 * smem, s>>>(a, vec); break;
        case 2: k_gram_planes<2><<<grid, 256, 2 * smem, s>>>(a, vec); break;
        default: k_gram_planes<1><<<grid, 256, 2 * smem, s>>>(a, vec); break;
      }
      return cudaGetLastError();
    }
  }
  cudaError_t oe = R == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_tile<T, 4>, 256, smem)
                 : R == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_tile<T, 2>, 256, smem)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_tile<T, 1>, 256, smem);
  if (oe != cudaSuccess) return oe;
  per_sm = std::max(per_sm, 1);
  const int grid = (int)std::min<long long>(items, (long long)num_sms * per_sm);
  switch (R) {
    case 4: k_gram_tile<T, 4><<<grid, 256, smem, s>>>(a); break;
    case 2: k_gram_tile<T, 2><<<grid, 256, smem, s>>>(a); break;
    default: k_gram_tile<T, 1><<<grid, 256, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_gram_f32(int N, int d, int nslots, const GramSource& src, unsigned int* out,
                            const PairFilter* filter, int num_sms, cudaStream_t s) {
  return launch_gram<float>(N, d, nslots, src, out, filter, num_sms, s);
}
cudaError_t launch_gram_f64(int N, int d, int nslots, const GramSource& src,
                            unsigned long long* out, int num_sms, cudaStream_t s) {
  return launch_gram<double>(N, d, nslots, src, out, nullptr, num_sms, s);
}

// ------------------------------------------------------------- init

__global__ void k_init_frame(int N, int d, uint64_t seed, double2* phi64, float2* phi32,
                             DevState* st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double* base = reinterpret_cast<double*>(phi64 + (size_t)j * d);
  const bool ok = gen_column<double>(nullptr, d, j, seed, 0u, 0u, 1u, 0.0, base, base + 1, 2);
  if (!ok && st) atomicOr(&st->error, (uint32_t)kErrZeroColumn);
  for (int i = 0; i < d; ++i) {
    const double2 v = phi64[(size_t)j * d + i];
    phi32[(size_t)j * d + i] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t launch_init_frame(int N, int d, uint64_t seed, double2* phi64, float2* phi32,
                              DevState* st, cudaStream_t s) {
  k_init_frame<<<(N + 127) / 128, 128, 0, s>>>(N, d, seed, phi64, phi32, st);
  return cudaGetLastError();
}

// ---------------------------------------------------- iteration start

__global__ void k_iter_begin(DevState* st, void* z0, size_t b0, void* z1, size_t b1, void* z2,
                             size_t b2, uint32_t call_iters) {
  __shared__ uint32_t act;
  if (threadIdx.x == 0) {
    if (call_iters) {
      // the first iteration of a call: its stop and its start counters
      const unsigned long long stop = (unsigned long long)st->t + call_iters;
      st->t_stop = stop > 0xffffffffull ? 0xffffffffu : (uint32_t)stop;
      st->t_call = st->t;
      st->accepts_call = st->accepts;
    }
    act = (!st->done && st->t < st->t_stop) ? 1u : 0u;
    st->active = act;
    st->npairs = 0u;
    st->overflow = 0u;
    st->use_screen = 0u;
    st->use_full = 0u;
    st->certify = 0u;
    if (act) {
      st->delta_used = st->delta;
      st->accepted = 0u;
      const bool scr = st->delta >= st->screen_min_delta;
      st->use_screen = scr ? 1u : 0u;
      st->use_full = scr ? 0u : 1u;
    }
  }
  __syncthreads();
  if (!act) return;
  void* ptrs[3] = {z0, z1, z2};
  size_t bytes[3] = {b0, b1, b2};
  for (int q = 0; q < 3; ++q) {
    if (!ptrs[q]) continue;
    uint32_t* p = reinterpret_cast<uint32_t*>(ptrs[q]);
    const size_t n = bytes[q] / 4;
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) p[e] = 0u;
  }
}

cudaError_t launch_iter_begin(DevState* st, void* zero0, size_t bytes0, void* zero1,
                              size_t bytes1, void* zero2, size_t bytes2, cudaStream_t s,
                              uint32_t call_iters) {
  k_iter_begin<<<1, 1024, 0, s>>>(st, zero0, bytes0, zero1, bytes1, zero2, bytes2, call_iters);
  return cudaGetLastError();
}

// ------------------------------------------------ the accept/radius rule

__device__ void apply_rule_and_trace(DevState* st, uint32_t cstar, double mu2_best,
                                     double mu2_screen, TraceRowDev* trace,
                                     uint32_t extra_flags = 0u) {
  const uint32_t t = st->t + 1u;
  const double dused = st->delta_used;
  const bool accept = mu2_best < st->mu2_cur;
  double dl;
  if (accept) {
    st->mu2_cur = mu2_best;
    dl = fmin(st->gamma_inc * dused, st->delta_max);
    st->accepts += 1u;
  } else {
    dl = fmax(st->gamma_dec * dused, st->delta_min);
  }
  st->delta = dl;
  st->accepted = accept ? 1u : 0u;
  st->cstar = cstar;
  st->mu2_best = mu2_best;
  st->mu2_screen = mu2_screen;
  st->t = t;
  if (st->mu2_cur <= st->target2) st->done = 1u;
  if (trace && st->trace_cap) {
    TraceRowDev& r = trace[(t - 1u) % st->trace_cap];
    r.t = t; r.cstar = cstar; r.mu2_best = mu2_best; r.mu2_screen = mu2_screen;
    r.mu2_cur = st->mu2_cur; r.delta_used = dused; r.delta_next = dl;
    r.accepted = accept ? 1 : 0; r.flags = (int32_t)((st->use_screen & 1u) | extra_flags);
  }
}

// argmin over candidates (lowest c on ties) then the rule; one CTA.
template <typename B>
__global__ void k_select_decide(DevState* st, const B* mu2, int K, TraceRowDev* trace) {
  if (!st->active) return;
  __shared__ B sv[32];
  __shared__ int sc[32];
  B bv = ~B(0);
  int bc = 0x7fffffff;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const B v = mu2[c];
    if (v < bv || (v == bv && c < bc)) { bv = v; bc = c; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const B ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
    if (ov < bv || (ov == bv && oc < bc)) { bv = ov; bc = oc; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = bv; sc[threadIdx.x >> 5] = bc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] < bv || (sv[w] == bv && sc[w] < bc)) { bv = sv[w]; bc = sc[w]; }
    const double m = (double)nonneg_from_bits(bv);
    apply_rule_and_trace(st, (uint32_t)bc, m, m, trace);
  }
}

cudaError_t launch_select_decide_f32(DevState* st, const unsigned int* mu2, int K,
                                     TraceRowDev* trace, cudaStream_t s) {
  k_select_decide<unsigned int><<<1, 1024, 0, s>>>(st, mu2, K, trace);
  return cudaGetLastError();
}
cudaError_t launch_select_decide_f64(DevState* st, const unsigned long long* mu2, int K,
                                     TraceRowDev* trace, cudaStream_t s) {
  k_select_decide<unsigned long long><<<1, 1024, 0, s>>>(st, mu2, K, trace);
  return cudaGetLastError();
}

// Regenerate the accepted candidate in place (one thread per column).  The
// counters are those of the iteration just decided: t = st->t.
template <typename T, typename O>
__global__ void k_commit(int N, int d, uint64_t seed, DevState* st,
                         typename Cplx<T>::type* phi, typename Cplx<O>::type* other) {
  if (!st->active || !st->accepted) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  T* base = reinterpret_cast<T*>(phi + (size_t)j * d);
  gen_column<T>(phi, d, j, seed, st->cstar, st->t, 0u, (T)st->delta_used, base, base + 1, 2);
  for (int i = 0; i < d; ++i) {
    const auto v = phi[(size_t)j * d + i];
    other[(size_t)j * d + i].x = (O)v.x;
    other[(size_t)j * d + i].y = (O)v.y;
  }
}

cudaError_t launch_commit_f32(int N, int d, uint64_t seed, DevState* st, float2* phi32,
                              double2* phi64, cudaStream_t s) {
  k_commit<float, double><<<(N + 127) / 128, 128, 0, s>>>(N, d, seed, st, phi32, phi64);
  return cudaGetLastError();
}
cudaError_t launch_commit_f64(int N, int d, uint64_t seed, DevState* st, double2* phi64,
                              float2* phi32, cudaStream_t s) {
  k_commit<double, float><<<(N + 127) / 128, 128, 0, s>>>(N, d, seed, st, phi64, phi32);
  return cudaGetLastError();
}

// ----------------------------------------------------------- screen mode

// The k smallest screen scores, ordered by (mu^2, c); one CTA.
// Ranked by the binary32 Gram of every candidate (not the screen), the
// survivors' binary32 scores are known already and are copied into mu2_top
// (the re-score pass, gated on use_screen, then does not run): the values are
// bit-identical to a re-score, which runs the same pair arithmetic.
// The k smallest keys (mu^2 bits << 32 | candidate), in increasing order: each
// warp extracts its own k smallest keys by k rounds of warp minima above the
// previous one (no CTA barrier), then warp 0 does the same over the warps'
// lists.  Keys are unique, so the result is the k smallest of all K.
constexpr int kTopkMax = 64;
__global__ void k_topk(DevState* st, const unsigned int* mu2, int K, int k, uint32_t* topk,
                       unsigned int* mu2_top) {
  if (!st->active) return;
  __shared__ unsigned long long cand[32 * kTopkMax];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long floor_key = 0ull;
  for (int r = 0; r < k; ++r) {
    unsigned long long best = ~0ull;
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
      const unsigned long long key = ((unsigned long long)mu2[c] << 32) | (unsigned)c;
      if ((r == 0 || key > floor_key) && key < best) best = key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      best = ov < best ? ov : best;
    }
    if (lane == 0) cand[warp * k + r] = best;
    floor_key = best;
  }
  __syncthreads();
  if (warp != 0) return;
  const int n = nw * k;
  floor_key = 0ull;
  for (int r = 0; r < k; ++r) {
    unsigned long long best = ~0ull;
    for (int q = lane; q < n; q += 32) {
      const unsigned long long key = cand[q];
      if ((r == 0 || key > floor_key) && key < best) best = key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      best = ov < best ? ov : best;
    }
    if (lane == 0) {
      topk[r] = (uint32_t)(best & 0xffffffffull);
      if (!st->use_screen) mu2_top[r] = (unsigned int)(best >> 32);
    }
    floor_key = best;
  }
}

// The same k smallest keys for K <= 1024 without rounds over the block:
// every thread holds one key ((score bits << 32) | c, all distinct); each warp
// sorts its 32 keys with a register bitonic network (shuffles) and keeps its k
// smallest, sorted, in shared memory; warp 0 then merges the 32 sorted lists,
// one list per lane, by k rounds of a warp minimum over the lists' heads.
constexpr int kSortMax = 1024;
__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
  return ((unsigned long long)hi << 32) | lo;
}
__global__ void __launch_bounds__(1024) k_topk_sort(DevState* st, const unsigned int* mu2, int K,
                                                    int k, uint32_t* topk, unsigned int* mu2_top) {
  if (!st->active) return;
  __shared__ unsigned long long lists[32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, c = threadIdx.x;
  unsigned long long key = c < K ? (((unsigned long long)mu2[c] << 32) | (unsigned)c) : ~0ull;
  // ascending bitonic sort of the warp's 32 keys, lane order
#pragma unroll
  for (int w = 2; w <= 32; w <<= 1) {
#pragma unroll
    for (int j = w >> 1; j > 0; j >>= 1) {
      const unsigned long long o = shfl_xor_u64(key, j);
      const bool lower = (lane & j) == 0, up = (lane & w) == 0;
      key = (lower == up) ? (o < key ? o : key) : (o > key ? o : key);
    }
  }
  if (lane < k) lists[warp][lane] = key;     // k <= 32
  __syncthreads();
  if (warp != 0) return;
  const int nw = (min(K, 1024) + 31) >> 5;
  int head = 0;
  for (int r = 0; r < k; ++r) {
    const unsigned long long mine = (lane < nw && head < k) ? lists[lane][head] : ~0ull;
    unsigned long long best = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = shfl_xor_u64(best, o);
      best = ov < best ? ov : best;
    }
    if (mine == best) ++head;            // keys are distinct: exactly one lane pops
    if (lane == 0) {
      topk[r] = (uint32_t)(best & 0xffffffffull);
      if (!st->use_screen) mu2_top[r] = (unsigned int)(best >> 32);
    }
  }
}

cudaError_t launch_topk(DevState* st, const unsigned int* mu2_screen, int K, int k,
                        uint32_t* topk, unsigned int* mu2_top, cudaStream_t s) {
  if (K <= kSortMax && k <= 32) k_topk_sort<<<1, 1024, 0, s>>>(st, mu2_screen, K, k, topk, mu2_top);
  else k_topk<<<1, 1024, 0, s>>>(st, mu2_screen, K, k, topk, mu2_top);
  return cudaGetLastError();
}

// Best survivor by its binary32 score (ties: lowest c), regenerated in
// binary64 from the binary64 frame, plus its binary32 rounding.
__global__ void k_materialize64(int N, int d, uint64_t seed, DevState* st,
                                const uint32_t* topk, const unsigned int* mu2_top, int k,
                                const double2* phi64, double2* cand64, float2* cand32,
                                unsigned int* hint_out, const uint32_t* list_count,
                                uint32_t list_cap, uint32_t* sel, int filter_available) {
  if (!st->active) return;
  unsigned int bv = mu2_top[0];
  uint32_t bc = topk[0];
  int bs = 0;
  for (int s = 1; s < k; ++s) {
    const unsigned int v = mu2_top[s];
    if (v < bv || (v == bv && topk[s] < bc)) { bv = v; bc = topk[s]; bs = s; }
  }
  // certify only a survivor the exact rule could accept
  const double m32 = (double)__uint_as_float(bv);
  const bool cert = !(m32 > st->mu2_cur + certify_margin_mu2(d));
  // one warp per column
  const int lane = threadIdx.x & 31;
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->cstar = bc;
    st->mu2_screen = m32;
    st->certify = cert ? 1u : 0u;
    if (hint_out && cert) *hint_out = bv;
    if (sel) {
      // the winner's pair list from the survivor pair pass, when complete,
      // holds every pair the certification needs; otherwise the binary32
      // filter pass runs, or without one the full binary64 pass
      sel[0] = (uint32_t)bs;
      const bool listed = st->use_screen && list_count[bs] <= list_cap;
      const bool need = cert && !listed;
      sel[1] = (need && filter_available) ? 1u : 0u;
      if (need && !filter_available) st->overflow = 1u;
    }
  }
  if (!cert || j >= N) return;
  const bool ok = gen_column_warp<double>(phi64, d, j, seed, bc, st->t + 1u, 0u, st->delta_used,
                                          cand64, lane);
  if (!ok && lane == 0) atomicOr(&st->error, (uint32_t)kErrZeroColumn);
  __syncwarp();
  for (int i = lane; i < d; i += 32) {
    const double2 v = cand64[(size_t)j * d + i];
    cand32[(size_t)j * d + i] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t launch_materialize64(int N, int d, uint64_t seed, DevState* st,
                                 const uint32_t* topk, const unsigned int* mu2_top, int k,
                                 const double2* phi64, double2* cand64, float2* cand32,
                                 cudaStream_t s, unsigned int* hint_out,
                                 const uint32_t* list_count, uint32_t list_cap, uint32_t* sel,
                                 bool filter_available) {
  const size_t threads = (size_t)N * 32;
  k_materialize64<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
      N, d, seed, st, topk, mu2_top, k, phi64, cand64, cand32, hint_out, list_count, list_cap,
      sel, filter_available ? 1 : 0);
  return cudaGetLastError();
}

// binary32 |G_jk|^2 of each survivor's listed pairs from its drawn planes
// ([i][column], real then imaginary, 2 d N floats per survivor), maxed into
// mu2[s]: the chain over i and the rounding of MicroTile::step and pair_abs2,
// so every pair has the bits the binary32 tile pass gives it.  A survivor
// whose list overflowed (count above cap) is left to the full pass.
// Column j of candidate c (iteration t, radius delta) around the binary32 frame
// by one warp, with gen_column's bits: lane p < P draws entries 2p and 2p + 1
// (x0 and x1), every lane adds the squared entries in gen_column's order (i
// ascending, broadcast from their lanes), and each lane divides its entries
// by the norm.  P <= 32 (d <= 64).  Returns false for a zero column (entries
// zero, as gen_column leaves them).
__device__ __forceinline__ bool gen_column_warp_f32(const float2* phi, int d, int j, uint64_t seed,
                                                    uint32_t c, uint32_t t, float delta,
                                                    int lane, float2& x0, float2& x1) {
  const int P = (d + 1) >> 1;
  x0 = x1 = make_float2(0.f, 0.f);
  if (lane < P) {
    const PhiloxOut u = philox4x32_10((uint32_t)j * (uint32_t)P + (uint32_t)lane, c, t, 0u,
                                      seed_lo(seed), seed_hi(seed));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * lane + h;
      if (i < d) {
        float zr, zi;
        cn_draw<float>(u.x[2 * h], u.x[2 * h + 1], zr, zi);
        const float2 v = phi[(size_t)j * d + i];
        const float2 x = make_float2(add_rn(v.x, mul_rn(delta, zr)), add_rn(v.y, mul_rn(delta, zi)));
        if (h == 0) x0 = x; else x1 = x;
      }
    }
  }
  const float q0 = add_rn(mul_rn(x0.x, x0.x), mul_rn(x0.y, x0.y));
  const float q1 = add_rn(mul_rn(x1.x, x1.x), mul_rn(x1.y, x1.y));
  float sq = 0.f;
  for (int i = 0; i < d; ++i) sq = add_rn(sq, __shfl_sync(0xffffffffu, (i & 1) ? q1 : q0, i >> 1));
  if (!(sq > 0.f)) {
    x0 = x1 = make_float2(0.f, 0.f);
    return false;
  }
  const float nrm = sqrt_rn(sq);
  x0 = make_float2(div_rn(x0.x, nrm), div_rn(x0.y, nrm));
  x1 = make_float2(div_rn(x1.x, nrm), div_rn(x1.y, nrm));
  return true;
}

// gen_column_warp_f32 for d <= 32 with two columns per warp: the half-warp
// h = lane / 16 draws column `col` (its lanes' own), lane 16h + p taking the
// entries 2p and 2p + 1; each half sums its column's squared entries in
// gen_column's order from its own lanes.
__device__ __forceinline__ bool gen_column_halfwarp_f32(const float2* phi, int d, int col,
                                                        uint64_t seed, uint32_t c, uint32_t t,
                                                        float delta, int lane, float2& x0,
                                                        float2& x1) {
  const int P = (d + 1) >> 1;
  const int p = lane & 15, base = lane & 16;
  x0 = x1 = make_float2(0.f, 0.f);
  if (p < P) {
    const PhiloxOut u = philox4x32_10((uint32_t)col * (uint32_t)P + (uint32_t)p, c, t, 0u,
                                      seed_lo(seed), seed_hi(seed));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * p + h;
      if (i < d) {
        float zr, zi;
        cn_draw<float>(u.x[2 * h], u.x[2 * h + 1], zr, zi);
        const float2 v = phi[(size_t)col * d + i];
        const float2 x = make_float2(add_rn(v.x, mul_rn(delta, zr)), add_rn(v.y, mul_rn(delta, zi)));
        if (h == 0) x0 = x; else x1 = x;
      }
    }
  }
  const float q0 = add_rn(mul_rn(x0.x, x0.x), mul_rn(x0.y, x0.y));
  const float q1 = add_rn(mul_rn(x1.x, x1.x), mul_rn(x1.y, x1.y));
  float sq = 0.f;
  for (int i = 0; i < d; ++i)
    sq = add_rn(sq, __shfl_sync(0xffffffffu, (i & 1) ? q1 : q0, base + (i >> 1)));
  if (!(sq > 0.f)) {
    x0 = x1 = make_float2(0.f, 0.f);
    return false;
  }
  const float nrm = sqrt_rn(sq);
  x0 = make_float2(div_rn(x0.x, nrm), div_rn(x0.y, nrm));
  x1 = make_float2(div_rn(x1.x, nrm), div_rn(x1.y, nrm));
  return true;
}

__global__ void k_pairs32(DevState* st, const uint2* lists, const uint32_t* count,
                          uint32_t cap, int N, int d, const float2* phi, uint64_t seed,
                          const uint32_t* topk, unsigned int* mu2) {
  if (!st->active || !st->use_screen) return;
  // survivor blockIdx.y; one warp per listed pair draws the pair's two columns
  // (gen_column_warp_f32: the bits of the survivors' binary32 draw) and runs
  // the tile pass's chain over i on the entries broadcast from their lanes
  const int sv = blockIdx.y;
  const uint32_t n = count[sv];
  if (n > cap) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t c = topk[sv], t = st->t + 1u;
  const float delta = (float)st->delta_used;
  // d <= 32: lanes 0-15 draw column j and lanes 16-31 column k at once
  const bool halves = d <= 32;
  for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n; q += warps) {
    const uint2 jk = lists[(size_t)sv * cap + q];
    float2 a0, a1, b0, b1;
    int bbase;
    if (halves) {
      const int col = lane < 16 ? (int)jk.x : (int)jk.y;
      const bool ok = gen_column_halfwarp_f32(phi, d, col, seed, c, t, delta, lane, a0, a1);
      if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(&st->error, (uint32_t)kErrZeroColumn);
      b0 = a0; b1 = a1;
      bbase = 16;
    } else {
      const bool okj = gen_column_warp_f32(phi, d, (int)jk.x, seed, c, t, delta, lane, a0, a1);
      const bool okk = gen_column_warp_f32(phi, d, (int)jk.y, seed, c, t, delta, lane, b0, b1);
      if ((!okj || !okk) && lane == 0) atomicOr(&st->error, (uint32_t)kErrZeroColumn);
      bbase = 0;
    }
    float gr = 0.f, gi = 0.f;
    for (int i = 0; i < d; ++i) {
      const int src = i >> 1;
      const bool odd = (i & 1) != 0;
      const float ar = __shfl_sync(0xffffffffu, odd ? a1.x : a0.x, src);
      const float ai = __shfl_sync(0xffffffffu, odd ? a1.y : a0.y, src);
      const float br = __shfl_sync(0xffffffffu, odd ? b1.x : b0.x, bbase + src);
      const float bi = __shfl_sync(0xffffffffu, odd ? b1.y : b0.y, bbase + src);
      gr = fmaf(ar, br, fmaf(ai, bi, gr));
      gi = fmaf(ar, bi, fmaf(-ai, br, gi));
    }
    if (lane == 0) atomic_max_nonneg(mu2 + sv, pair_abs2(gr, gi));
  }
}

cudaError_t launch_pairs32(DevState* st, const uint2* lists, const uint32_t* count,
                           uint32_t cap, int k, int N, int d, const float2* phi, uint64_t seed,
                           const uint32_t* topk, unsigned int* mu2, cudaStream_t s) {
  if (d > 64) return cudaErrorInvalidValue;
  const unsigned bx = std::min(16u, (cap + 7) / 8);
  k_pairs32<<<dim3(bx, (unsigned)k), 256, 0, s>>>(st, lists, count, cap, N, d, phi, seed, topk,
                                                  mu2);
  return cudaGetLastError();
}

// |G| in binary32 of a frame rounded from binary64 differs from the binary64
// |G| by at most ~(2 + 2 (2d)) u, u = 2^-24 (rounding of the entries plus a
// 2d-term dot product per part); twice a generous 4x of that bound separates
// "can be the maximum" from "cannot".
float certify_margin(int d) { return (float)(8.0 * (2.0 * d + 2.0) * std::ldexp(1.0, -24)); }

// Binary64 mu^2 of a normalised frame (p64, and p32 its binary32 rounding)
// into *cert64: the binary32 maximum (cert32[0]), the pairs within the
// binary32 / binary64 margin of it (filter pass into cert32[1] and pairs),
// those pairs in binary64, and all pairs in binary64 when the list
// overflowed.  cert32[0..1], *cert64, *npairs and *overflow start at zero.
// Every certified mu^2 of the precision form comes from these passes (or the
// iteration's own pair lists), so a frame has one certified value whatever
// entry point scores it.
cudaError_t launch_frame_certify(int N, int d, const double2* p64, const float2* p32,
                                 unsigned int* cert32, unsigned long long* cert64, uint2* pairs,
                                 uint32_t cap, uint32_t* npairs, uint32_t* overflow,
                                 const uint32_t* active, int num_sms, cudaStream_t s) {
  GramSource src{};
  src.perturb = false;
  src.phi = p32;
  src.normalize = false;
  src.gate = active;
  // one binary32 pass: the max into cert32[0] and, tile by tile, the pairs
  // within the margin of the tile's maximum
  PairFilter pf{nullptr, certify_margin(d), pairs, npairs, cap, overflow, nullptr, 0.f, 1};
  cudaError_t e = launch_gram_f32(N, d, 1, src, cert32, &pf, num_sms, s);
  if (e != cudaSuccess) return e;
  if ((e = launch_pairs64(active, npairs, pairs, cap, d, p64, cert64, s)) != cudaSuccess) return e;
  GramSource full{};
  full.perturb = false;
  full.phi = p64;
  full.normalize = false;
  full.gate = overflow;
  return launch_gram_f64(N, d, 1, full, cert64, num_sms, s);
}

// binary64 |G_jk|^2 of columns x and y (d entries each) by one warp: lane l
// accumulates entries l, l + 32, .. (each part two fused multiply-adds, as in
// the tile passes), and the lanes' partial sums meet in a butterfly of
// additions, which leaves the same bits in every lane (a + b = b + a).  Every
// binary64 pair kernel of the precision form uses it, so a pair has one value
// whatever kernel evaluates it; the dependent chain is 2 d / 32 fused
// multiply-adds and five additions instead of 2 d (binary64 latency is long
// on this GPU).
__device__ __forceinline__ double pair_abs2_warp64(const double2* x, const double2* y, int d,
                                                   int lane) {
  double re = 0.0, im = 0.0;
  for (int i = lane; i < d; i += 32) {
    const double2 u = x[i], v = y[i];
    re = fma(u.x, v.x, fma(u.y, v.y, re));
    im = fma(u.x, v.y, fma(-u.y, v.x, im));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  return pair_abs2(re, im);
}

// binary64 |G_jk|^2 of the preselected pairs, one warp per pair.
__global__ void k_pairs64(const uint32_t* active, const uint32_t* npairs, const uint2* pairs,
                          uint32_t cap, int d, const double2* f, unsigned long long* out,
                          const unsigned int* hint_bits, const unsigned int* own_bits,
                          float hint_slack_mu2, uint32_t* overflow, const uint32_t* sel,
                          const uint2* lists, const uint32_t* list_count, uint32_t list_cap) {
  if (active && !*active) return;
  uint32_t n;
  if (sel && sel[1] == 0u) {
    // the winner's list from the survivor pair pass (complete: see k_materialize64)
    const uint32_t w = sel[0];
    pairs = lists + (size_t)w * list_cap;
    n = min(list_count[w], list_cap);
  } else {
    if (hint_bits && blockIdx.x == 0 && threadIdx.x == 0 &&
        fmaxf(__uint_as_float(*hint_bits) - hint_slack_mu2, 0.0f) > __uint_as_float(*own_bits))
      atomicExch(overflow, 1u);
    n = min(*npairs, cap);
  }
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  double m = 0.0;
  for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    const uint2 jk = pairs[p];
    m = fmax(m, pair_abs2_warp64(f + (size_t)jk.x * d, f + (size_t)jk.y * d, d, lane));
  }
  if (lane == 0 && m > 0.0) atomic_max_nonneg(out, m);
}

cudaError_t launch_pairs64(const uint32_t* active, const uint32_t* npairs, const uint2* pairs,
                           uint32_t cap, int d, const double2* frame64, unsigned long long* out,
                           cudaStream_t s, const unsigned int* hint_bits,
                           const unsigned int* own_bits, float hint_slack_mu2,
                           uint32_t* overflow, const uint32_t* sel, const uint2* lists,
                           const uint32_t* list_count, uint32_t list_cap) {
  k_pairs64<<<256, 256, 0, s>>>(active, npairs, pairs, cap, d, frame64, out, hint_bits, own_bits,
                               hint_slack_mu2, overflow, sel, lists, list_count, list_cap);
  return cudaGetLastError();
}

// The rule and the commit of the certified (or bound-rejected) survivor in one
// launch: every CTA forms the same decision from the state as the iteration
// left it and copies its share of the candidate when it is accepted; the last
// CTA to finish (counter *done, reset by that CTA) then applies the rule and
// writes the trace row, so no CTA reads the state after it changed.
__global__ void k_decide_commit(size_t n, DevState* st, const unsigned long long* mu2_64,
                                TraceRowDev* trace, const double2* cand64, const float2* cand32,
                                double2* phi64, float2* phi32, unsigned int* done) {
  if (!st->active) return;
  const bool cert = st->certify != 0u;
  const double best = cert ? nonneg_from_bits(*mu2_64) : st->mu2_screen;
  if (best < st->mu2_cur) {   // the rule's acceptance test
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x) {
      phi64[e] = cand64[e];
      phi32[e] = cand32[e];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1u) {
      *done = 0u;
      __threadfence();
      // uncertified: the survivor's binary32 score is above the current mu^2
      // by more than the error bound, and the rule rejects it on that value
      apply_rule_and_trace(st, st->cstar, best, st->mu2_screen, trace,
                           (cert ? 0u : 2u) | (st->overflow ? 4u : 0u));
    }
  }
}

cudaError_t launch_decide_commit(int N, int d, DevState* st, const unsigned long long* mu2_64,
                                 TraceRowDev* trace, const double2* cand64, const float2* cand32,
                                 double2* phi64, float2* phi32, unsigned int* done,
                                 cudaStream_t s) {
  const size_t n = (size_t)N * d;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 1024);
  k_decide_commit<<<grid, 256, 0, s>>>(n, st, mu2_64, trace, cand64, cand32, phi64, phi32, done);
  return cudaGetLastError();
}

// ---------------------------------------------------------- utilities

__global__ void k_normalize64(int N, int d, const double2* in, double2* out64, float2* out32,
                              DevState* st) {
  // one warp per column; in and out64 may alias
  const int lane = threadIdx.x & 31;
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (j >= N) return;
  const double2* col = in + (size_t)j * d;
  double s = 0.0;
  for (int i = lane; i < d; i += 32) s += col[i].x * col[i].x + col[i].y * col[i].y;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (!(s > 0.0)) {
    if (st && lane == 0) atomicOr(&st->error, (uint32_t)kErrZeroColumn);
    return;
  }
  const double nrm = sqrt(s);
  for (int i = lane; i < d; i += 32) {
    const double2 v = col[i];
    const double2 w = make_double2(v.x / nrm, v.y / nrm);
    out64[(size_t)j * d + i] = w;
    out32[(size_t)j * d + i] = make_float2((float)w.x, (float)w.y);
  }
}

cudaError_t launch_normalize64(int N, int d, const double2* in, double2* out64, float2* out32,
                               DevState* st, cudaStream_t s) {
  const size_t threads = (size_t)N * 32;
  k_normalize64<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(N, d, in, out64, out32, st);
  return cudaGetLastError();
}

__global__ void k_gen_candidate(int N, int d, uint64_t seed, uint32_t t, uint32_t c,
                                double delta, bool f64, const double2* phi64,
                                const float2* phi32, double2* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double* base = reinterpret_cast<double*>(out + (size_t)j * d);
  if (f64) {
    gen_column<double>(phi64, d, j, seed, c, t, 0u, delta, base, base + 1, 2);
  } else {
    // binary32 generation into a scratch of the output, then widened
    float* fb = reinterpret_cast<float*>(base);
    gen_column<float>(phi32, d, j, seed, c, t, 0u, (float)delta, fb, fb + 1, 2);
    for (int i = d - 1; i >= 0; --i) {
      const float re = fb[2 * i], im = fb[2 * i + 1];
      base[2 * i] = (double)re;
      base[2 * i + 1] = (double)im;
    }
  }
}

cudaError_t launch_gen_candidate(int N, int d, uint64_t seed, uint32_t t, uint32_t c,
                                 double delta, bool f64, const double2* phi64,
                                 const float2* phi32, double2* out, cudaStream_t s) {
  k_gen_candidate<<<(N + 127) / 128, 128, 0, s>>>(N, d, seed, t, c, delta, f64, phi64, phi32,
                                                   out);
  return cudaGetLastError();
}

// ------------------------------------------------------ batched searches
//
// Many independent instances advance together: each kernel below covers all
// of them in one launch.  Every instance keeps its own DevState and
// counters, so its trajectory is the one it would follow alone.

template <typename B>
__global__ void k_batch_begin(SlotDesc* slots, int n, unsigned long long* counters, int ncounters,
                              int screen_mode) {
  const int s = blockIdx.x;
  if (s == 0 && threadIdx.x < ncounters) counters[threadIdx.x] = 0ull;
  if (s >= n) return;
  const SlotDesc& sd = slots[s];
  DevState* st = sd.st;
  __shared__ uint32_t act;
  if (threadIdx.x == 0) {
    act = (!st->done && st->t < st->t_stop) ? 1u : 0u;
    st->active = act;
    st->npairs = 0u;
    st->overflow = 0u;
    st->certify = 0u;
    const bool scr = act && screen_mode && sd.screen && st->delta >= st->screen_min_delta;
    st->use_screen = scr ? 1u : 0u;
    st->use_full = (act && !scr) ? 1u : 0u;
    if (act) {
      st->delta_used = st->delta;
      st->accepted = 0u;
    }
  }
  __syncthreads();
  if (!act) return;
  B* mu2 = reinterpret_cast<B*>(sd.mu2);
  for (int c = threadIdx.x; c < sd.K; c += blockDim.x) mu2[c] = B(0);
  if (screen_mode) {
    for (int c = threadIdx.x; c < sd.topk_n; c += blockDim.x) sd.mu2_top[c] = 0u;
    if (threadIdx.x == 0) { sd.cert32[0] = 0u; sd.cert32[1] = 0u; *sd.cert64 = 0ull; }
  }
}

cudaError_t launch_batch_begin(SlotDesc* slots, int n, unsigned long long* counters, int ncounters,
                               bool f64, bool screen_mode, cudaStream_t s) {
  const int grid = n > 0 ? n : 1;
  if (f64) k_batch_begin<unsigned long long><<<grid, 256, 0, s>>>(slots, n, counters, ncounters, screen_mode);
  else k_batch_begin<unsigned int><<<grid, 256, 0, s>>>(slots, n, counters, ncounters, screen_mode);
  return cudaGetLastError();
}

// Persistent scoring pass: CTAs take work items (instance, k, tile) from
// *counter until nitems are done.  group lists the instances of this tile
// width in the order of their items; group_begin[g] is the first item of
// group[g] (group_begin[ngroup] = nitems).  What an item is depends on the
// pass (BatchPassMode): a candidate (k = candidate index, or the k-th top-k
// survivor) generated around the instance's frame, or the instance's stored
// winner frame (one item per tile).
template <typename T, int R>
__global__ void __launch_bounds__(256, TileCtas<T>::value) k_batch_score(const SlotDesc* slots, const int* group,
                                                     const long long* group_begin, int ngroup,
                                                     long long nitems,
                                                     unsigned long long* counter, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[8];
  __shared__ int zero_col;
  __shared__ long long item;
  T* sm = reinterpret_cast<T*>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long w = item;
    if (w >= nitems) return;
    // instance of this item: last g with group_begin[g] <= w
    int lo = 0, hi = ngroup - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (group_begin[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const SlotDesc& sd = slots[group[lo]];
    const DevState* st = sd.st;
    bool run;
    switch (mode) {
      case kPassFull: run = st->active && st->use_full; break;
      case kPassRescore: run = st->active && st->use_screen; break;
      case kPassFrame64: run = st->active && st->overflow; break;
      default: run = st->active && st->certify; break;   // FrameMax, Filter
    }
    if (run) {
      // tiles at this launch's width (the binary64 frame pass may run an
      // instance narrower than its ranking width)
      const int nbw = (sd.N + 16 * R - 1) / (16 * R);
      const long long ntw = (long long)nbw * (nbw + 1) / 2;
      const long long local = w - group_begin[lo];
      const int k = (int)(local / ntw);
      TileItem it;
      it.N = sd.N; it.d = sd.d;
      tile_coords((int)(local - (long long)k * ntw), it.I, it.J);
      it.normalize = false;
      it.seed = sd.seed;
      it.t = st->t + 1u;
      it.delta = st->delta_used;
      T thr = T(-1);
      PairFilter pf{};   // every field zero until set below (local = 0)
      const PairFilter* filter = nullptr;
      if (mode == kPassFull || mode == kPassRescore) {
        it.perturb = true;
        it.phi = sd.phi;
        it.c = mode == kPassFull ? (uint32_t)k : sd.topk[k];
      } else {
        it.perturb = false;
        it.c = 0u;
        it.phi = mode == kPassFrame64 ? (const void*)sd.cand64 : (const void*)sd.cand32;
        if (mode == kPassFilter) {
          pf.mu2_ref = &sd.cert32[0];
          pf.margin = (float)(8.0 * (2.0 * sd.d + 2.0) / 16777216.0);
          pf.pairs = sd.pairs;
          pf.npairs = &const_cast<DevState*>(st)->npairs;
          pf.cap = sd.pair_cap;
          pf.overflow = &const_cast<DevState*>(st)->overflow;
          pf.scale_bits = nullptr;
          // cert32[0] is the chosen survivor's binary32 score, within the
          // fp32 / fp64 bound of this frame's binary32 max (checked by the
          // pair pass, which falls back to the full binary64 pass)
          pf.ref_slack_mu2 = (float)certify_margin_mu2(sd.d);
          const float lo2 = filter_lo(pf);
          thr = (T)(lo2 * lo2);
          filter = &pf;
        }
      }
      if (threadIdx.x == 0) zero_col = 0;
      T m = score_tile<T, R>(it, sm, &zero_col, thr, filter);
      if (zero_col && threadIdx.x == 0)
        atomicOr(&const_cast<DevState*>(st)->error, (uint32_t)kErrZeroColumn);
      m = block_max<T>(m, red);
      if (threadIdx.x == 0) {
        typename Mu2Bits<T>::type* out;
        switch (mode) {
          case kPassFull: out = reinterpret_cast<typename Mu2Bits<T>::type*>(sd.mu2) + k; break;
          case kPassRescore: out = reinterpret_cast<typename Mu2Bits<T>::type*>(sd.mu2_top) + k; break;
          case kPassFrameMax: out = reinterpret_cast<typename Mu2Bits<T>::type*>(sd.cert32); break;
          case kPassFilter: out = reinterpret_cast<typename Mu2Bits<T>::type*>(sd.cert32 + 1); break;
          default: out = reinterpret_cast<typename Mu2Bits<T>::type*>(sd.cert64); break;
        }
        atomic_max_nonneg(out, m);
      }
    }
    __syncthreads();
  }
}

// Whole-candidate scoring for small instances (batched form).  The CTA draws
// all N columns of candidate c once into shared memory as [i][column] planes
// (the tile path draws every column block once per tile of its row and
// column), then reduces every pair j < k with 4 x 4 micro-tiles spread over
// the threads.  Generation (gen_candidate_cta: gen_column's arithmetic with
// the draws spread over the CTA), the sequential chain over i and the explicit
// rounding of |G|^2 are those of score_tile, so the scores are the same bits.
// Np = N rounded up to a multiple of 4; padded columns are zero.
template <typename T>
__device__ T score_resident(int N, int d, const void* phi, uint64_t seed, uint32_t c, uint32_t t,
                            double delta, T* sm, int* zero_col) {
  using C = typename Cplx<T>::type;
  const int Np = (N + 3) & ~3;
  T* sRe = sm;
  T* sIm = sm + (size_t)d * Np;
  __syncthreads();
  for (int q = threadIdx.x; q < (Np - N) * d; q += blockDim.x) {   // padded columns
    const int j = N + q / d, i = q % d;
    sRe[i * Np + j] = T(0);
    sIm[i * Np + j] = T(0);
  }
  gen_candidate_cta<T>(reinterpret_cast<const C*>(phi), N, d, seed, c, t, (T)delta, sRe, sIm, Np,
                       zero_col);
  const int nq = Np >> 2;
  const int nmt = nq * (nq + 1) / 2;
  T m = T(0);
  for (int w = threadIdx.x; w < nmt; w += blockDim.x) {
    int a, b;
    tile_coords(w, a, b);   // a <= b: rows 4a.., columns 4b..
    MicroTile<T, 4> acc;
    acc.zero();
    for (int i = 0; i < d; ++i) {
      const T* ri = sRe + (size_t)i * Np;
      const T* ii = sIm + (size_t)i * Np;
      T ar[4], ai[4], br[4], bi[4];
      load_run<T, 4>(ri + 4 * a, ar);
      load_run<T, 4>(ii + 4 * a, ai);
      load_run<T, 4>(ri + 4 * b, br);
      load_run<T, 4>(ii + 4 * b, bi);
      acc.step(ar, ai, br, bi);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int j = 4 * a + x, k = 4 * b + y;
        if (j < k && k < N) m = fmax(m, pair_abs2(acc.get_re(x, y), acc.get_im(x, y)));
      }
  }
  return m;
}

template <typename T>
size_t resident_smem(int d, int N) {
  return (size_t)2 * d * (size_t)((N + 3) & ~3) * sizeof(T);
}

// Persistent whole-candidate pass over the resident instances of a batch:
// work items (instance, k) from *counter; k indexes the candidates (full
// ranking) or the top-k survivors (re-score), as in k_batch_score.
template <typename T>
__global__ void __launch_bounds__(128) k_batch_resident(const SlotDesc* slots, const int* group,
                                                        const long long* group_begin, int ngroup,
                                                        long long nitems,
                                                        unsigned long long* counter, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[4];
  __shared__ int zero_col;
  __shared__ long long item;
  T* sm = reinterpret_cast<T*>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long w = item;
    if (w >= nitems) return;
    int lo = 0, hi = ngroup - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (group_begin[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const SlotDesc& sd = slots[group[lo]];
    const DevState* st = sd.st;
    const bool run = st->active && (mode == kPassFull ? st->use_full : st->use_screen);
    if (run) {
      const int k = (int)(w - group_begin[lo]);
      const uint32_t c = mode == kPassFull ? (uint32_t)k : sd.topk[k];
      if (threadIdx.x == 0) zero_col = 0;
      T m = score_resident<T>(sd.N, sd.d, sd.phi, sd.seed, c, st->t + 1u, st->delta_used, sm,
                              &zero_col);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
        if (zero_col) atomicOr(&const_cast<DevState*>(st)->error, (uint32_t)kErrZeroColumn);
        typename Mu2Bits<T>::type* out =
            mode == kPassFull ? reinterpret_cast<typename Mu2Bits<T>::type*>(sd.mu2) + k
                              : reinterpret_cast<typename Mu2Bits<T>::type*>(sd.mu2_top) + k;
        atomic_max_nonneg(out, m);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_batch_resident(bool f64, const SlotDesc* slots, const int* group,
                                  const long long* group_begin, int ngroup, long long nitems,
                                  unsigned long long* counter, size_t smem, int grid,
                                  cudaStream_t s, int mode) {
  if (ngroup < 1 || nitems < 1) return cudaSuccess;
  if (mode != kPassFull && mode != kPassRescore) return cudaErrorInvalidValue;
  if (f64)
    k_batch_resident<double><<<grid, 128, smem, s>>>(slots, group, group_begin, ngroup, nitems,
                                                     counter, mode);
  else
    k_batch_resident<float><<<grid, 128, smem, s>>>(slots, group, group_begin, ngroup, nitems,
                                                    counter, mode);
  return cudaGetLastError();
}

size_t resident_smem_bytes(bool f64, int d, int N) {
  return f64 ? resident_smem<double>(d, N) : resident_smem<float>(d, N);
}

template <typename T>
static cudaError_t launch_batch_score_t(int R, const SlotDesc* slots, const int* group,
                                        const long long* group_begin, int ngroup, long long nitems,
                                        unsigned long long* counter, size_t smem, int grid,
                                        cudaStream_t s, int mode) {
  if (ngroup < 1 || nitems < 1) return cudaSuccess;
  switch (R) {
    case 4: k_batch_score<T, 4><<<grid, 256, smem, s>>>(slots, group, group_begin, ngroup, nitems, counter, mode); break;
    case 2: k_batch_score<T, 2><<<grid, 256, smem, s>>>(slots, group, group_begin, ngroup, nitems, counter, mode); break;
    case 1: k_batch_score<T, 1><<<grid, 256, smem, s>>>(slots, group, group_begin, ngroup, nitems, counter, mode); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_score(bool f64, int R, const SlotDesc* slots, const int* group,
                               const long long* group_begin, int ngroup, long long nitems,
                               unsigned long long* counter, size_t smem, int grid,
                               cudaStream_t s, int mode) {
  return f64 ? launch_batch_score_t<double>(R, slots, group, group_begin, ngroup, nitems, counter,
                                            smem, grid, s, mode)
             : launch_batch_score_t<float>(R, slots, group, group_begin, ngroup, nitems, counter,
                                           smem, grid, s, mode);
}

// Screen modes: the top_n smallest screen (or fp32) scores of each instance,
// ordered by (mu^2, c); one CTA per instance.
__global__ void k_batch_topk(SlotDesc* slots, int n) {
  const SlotDesc& sd = slots[blockIdx.x];
  if (!sd.st->active) return;
  const unsigned int* mu2 = reinterpret_cast<const unsigned int*>(sd.mu2);
  __shared__ unsigned long long sk[8];
  __shared__ unsigned long long last;
  if (threadIdx.x == 0) last = 0ull;
  __syncthreads();
  for (int r = 0; r < sd.topk_n; ++r) {
    const unsigned long long floor_key = last;
    unsigned long long best = ~0ull;
    for (int c = threadIdx.x; c < sd.K; c += blockDim.x) {
      const unsigned long long key = ((unsigned long long)mu2[c] << 32) | (unsigned)c;
      if ((r == 0 || key > floor_key) && key < best) best = key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      best = ov < best ? ov : best;
    }
    if ((threadIdx.x & 31) == 0) sk[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = sk[w] < best ? sk[w] : best;
      sd.topk[r] = (uint32_t)(best & 0xffffffffull);
      if (!sd.st->use_screen) sd.mu2_top[r] = (unsigned int)(best >> 32);
      last = best;
    }
    __syncthreads();
  }
}

cudaError_t launch_batch_topk(SlotDesc* slots, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  k_batch_topk<<<n, 256, 0, s>>>(slots, n);
  return cudaGetLastError();
}

// The best survivor of each instance regenerated in binary64 (one warp per
// column, instance = blockIdx.y), plus its binary32 rounding.
__global__ void k_batch_materialize64(SlotDesc* slots, int n) {
  const SlotDesc& sd = slots[blockIdx.y];
  DevState* st = sd.st;
  if (!st->active) return;
  unsigned int bv = sd.mu2_top[0];
  uint32_t bc = sd.topk[0];
  for (int q = 1; q < sd.topk_n; ++q) {
    const unsigned int v = sd.mu2_top[q];
    if (v < bv || (v == bv && sd.topk[q] < bc)) { bv = v; bc = sd.topk[q]; }
  }
  const double m32 = (double)__uint_as_float(bv);
  const bool cert = !(m32 > st->mu2_cur + certify_margin_mu2(sd.d));
  const int lane = threadIdx.x & 31;
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->cstar = bc;
    st->mu2_screen = m32;
    st->certify = cert ? 1u : 0u;
    if (cert) sd.cert32[0] = bv;   // the filter pass's hint (no separate max pass)
  }
  if (!cert || j >= sd.N) return;
  const double2* phi64 = reinterpret_cast<const double2*>(sd.phi_other);
  const bool ok = gen_column_warp<double>(phi64, sd.d, j, sd.seed, bc, st->t + 1u, 0u,
                                          st->delta_used, sd.cand64, lane);
  if (!ok && lane == 0) atomicOr(&st->error, (uint32_t)kErrZeroColumn);
  __syncwarp();
  for (int i = lane; i < sd.d; i += 32) {
    const double2 v = sd.cand64[(size_t)j * sd.d + i];
    sd.cand32[(size_t)j * sd.d + i] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t launch_batch_materialize64(SlotDesc* slots, int n, int maxN, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  dim3 grid((unsigned)(((size_t)maxN * 32 + 255) / 256), n);
  k_batch_materialize64<<<grid, 256, 0, s>>>(slots, n);
  return cudaGetLastError();
}

// binary64 |G|^2 over each instance's preselected pairs (one CTA per instance).
__global__ void k_batch_pairs64(SlotDesc* slots, int n) {
  const SlotDesc& sd = slots[blockIdx.x];
  const DevState* st = sd.st;
  if (!st->active || !st->certify) return;
  // the filter pass ran from the survivor's score as a hint: if the hint less
  // its slack exceeds the pass's own max, pairs may have been missed
  if (threadIdx.x == 0 &&
      fmaxf(__uint_as_float(sd.cert32[0]) - (float)certify_margin_mu2(sd.d), 0.0f) >
          __uint_as_float(sd.cert32[1]))
    atomicExch(&const_cast<DevState*>(st)->overflow, 1u);
  const uint32_t np = min(st->npairs, sd.pair_cap);
  const int d = sd.d, lane = threadIdx.x & 31;
  double m = 0.0;
  for (uint32_t p = threadIdx.x >> 5; p < np; p += blockDim.x >> 5) {
    const uint2 jk = sd.pairs[p];
    m = fmax(m, pair_abs2_warp64(sd.cand64 + (size_t)jk.x * d, sd.cand64 + (size_t)jk.y * d, d,
                                 lane));
  }
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_nonneg(sd.cert64, m);
}

cudaError_t launch_batch_pairs64(SlotDesc* slots, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  k_batch_pairs64<<<n, 256, 0, s>>>(slots, n);
  return cudaGetLastError();
}

__global__ void k_batch_decide_certified(SlotDesc* slots, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const SlotDesc& sd = slots[s];
  DevState* st = sd.st;
  if (!st->active) return;
  const bool cert = st->certify != 0u;
  apply_rule_and_trace(st, st->cstar, cert ? nonneg_from_bits(*sd.cert64) : st->mu2_screen,
                       st->mu2_screen, sd.trace, (cert ? 0u : 2u) | (st->overflow ? 4u : 0u));
}

cudaError_t launch_batch_decide_certified(SlotDesc* slots, int n, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  k_batch_decide_certified<<<(n + 127) / 128, 128, 0, s>>>(slots, n);
  return cudaGetLastError();
}

__global__ void k_batch_commit_copy(SlotDesc* slots, int n) {
  const SlotDesc& sd = slots[blockIdx.y];
  DevState* st = sd.st;
  if (!st->active || !st->accepted) return;
  const size_t nd = (size_t)sd.N * sd.d;
  double2* phi64 = reinterpret_cast<double2*>(sd.phi_other);
  float2* phi32 = reinterpret_cast<float2*>(sd.phi);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nd;
       e += (size_t)gridDim.x * blockDim.x) {
    phi64[e] = sd.cand64[e];
    phi32[e] = sd.cand32[e];
  }
}

cudaError_t launch_batch_commit_copy(SlotDesc* slots, int n, int maxN, int maxd, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const size_t nd = (size_t)maxN * maxd;
  dim3 grid((unsigned)std::min<size_t>((nd + 255) / 256, 64), n);
  k_batch_commit_copy<<<grid, 256, 0, s>>>(slots, n);
  return cudaGetLastError();
}

template <typename K>
static cudaError_t occupancy_of(K kernel, size_t smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kernel, 256, smem);
}

cudaError_t batch_resident_occupancy(bool f64, size_t smem, int* blocks_per_sm) {
  return f64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_resident<double>,
                                                             128, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_resident<float>,
                                                             128, smem);
}

cudaError_t batch_score_occupancy(bool f64, int R, size_t smem, int* blocks_per_sm) {
  if (f64) {
    if (R == 4) return occupancy_of(k_batch_score<double, 4>, smem, blocks_per_sm);
    if (R == 2) return occupancy_of(k_batch_score<double, 2>, smem, blocks_per_sm);
    return occupancy_of(k_batch_score<double, 1>, smem, blocks_per_sm);
  }
  if (R == 4) return occupancy_of(k_batch_score<float, 4>, smem, blocks_per_sm);
  if (R == 2) return occupancy_of(k_batch_score<float, 2>, smem, blocks_per_sm);
  return occupancy_of(k_batch_score<float, 1>, smem, blocks_per_sm);
}

size_t gram_smem_bytes(bool f64, int d, int R) {
  return f64 ? gram_smem<double>(d, R) : gram_smem<float>(d, R);
}

// argmin over each instance's K scores, then its accept/radius rule; one CTA each.
template <typename B>
__global__ void k_batch_decide(SlotDesc* slots, int n) {
  const int s = blockIdx.x;
  if (s >= n) return;
  DevState* st = slots[s].st;
  if (!st->active) return;
  const B* mu2 = reinterpret_cast<const B*>(slots[s].mu2);
  const int K = slots[s].K;
  __shared__ B sv[8];
  __shared__ int sc[8];
  B bv = ~B(0);
  int bc = 0x7fffffff;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const B v = mu2[c];
    if (v < bv || (v == bv && c < bc)) { bv = v; bc = c; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const B ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
    if (ov < bv || (ov == bv && oc < bc)) { bv = ov; bc = oc; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = bv; sc[threadIdx.x >> 5] = bc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] < bv || (sv[w] == bv && sc[w] < bc)) { bv = sv[w]; bc = sc[w]; }
    const double m = (double)nonneg_from_bits(bv);
    apply_rule_and_trace(st, (uint32_t)bc, m, m, slots[s].trace);
  }
}

cudaError_t launch_batch_decide(SlotDesc* slots, int n, bool f64, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  if (f64) k_batch_decide<unsigned long long><<<n, 256, 0, s>>>(slots, n);
  else k_batch_decide<unsigned int><<<n, 256, 0, s>>>(slots, n);
  return cudaGetLastError();
}

// Regenerate each accepted candidate in place (instance = blockIdx.y).
template <typename T, typename O>
__global__ void k_batch_commit(SlotDesc* slots, int n) {
  const SlotDesc& sd = slots[blockIdx.y];
  DevState* st = sd.st;
  if (!st->active || !st->accepted) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= sd.N) return;
  using C = typename Cplx<T>::type;
  using CO = typename Cplx<O>::type;
  C* phi = reinterpret_cast<C*>(sd.phi);
  CO* other = reinterpret_cast<CO*>(sd.phi_other);
  const int d = sd.d;
  T* base = reinterpret_cast<T*>(phi + (size_t)j * d);
  gen_column<T>(phi, d, j, sd.seed, st->cstar, st->t, 0u, (T)st->delta_used, base, base + 1, 2);
  for (int i = 0; i < d; ++i) {
    const C v = phi[(size_t)j * d + i];
    other[(size_t)j * d + i].x = (O)v.x;
    other[(size_t)j * d + i].y = (O)v.y;
  }
}

cudaError_t launch_batch_commit(SlotDesc* slots, int n, int maxN, bool f64, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  dim3 grid((maxN + 127) / 128, n);
  if (f64) k_batch_commit<double, float><<<grid, 128, 0, s>>>(slots, n);
  else k_batch_commit<float, double><<<grid, 128, 0, s>>>(slots, n);
  return cudaGetLastError();
}

template <typename K> static cudaError_t allow_max_dynamic_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

cudaError_t init_kernel_attributes() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_planes<4>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_planes<2>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_planes<1>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_tile<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_tile<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_tile<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_tile<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_tile<double, 2>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_gram_tile<double, 1>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_score<float, 4>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_score<float, 2>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_score<float, 1>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_score<double, 4>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_score<double, 2>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_score<double, 1>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_resident<float>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_batch_resident<double>, optin)) != cudaSuccess) return e;
  if ((e = allow_max_dynamic_smem(k_draw_planes_tiled_f32, optin)) != cudaSuccess) return e;
  if ((e = init_lse_attributes(optin)) != cudaSuccess) return e;
  if ((e = init_diag_attributes(optin)) != cudaSuccess) return e;
  return init_screen_attributes(optin);
}

}  // namespace trstmi
