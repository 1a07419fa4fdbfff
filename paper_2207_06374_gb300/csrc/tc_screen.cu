// bf16 tensor-core screen of the candidate Gram matrices (tcgen05, sm_103a).
//
// For candidate c of iteration t the CTA forms X = [A; B] (2*DP x N, bf16),
// the real split of Phi_c = normalise_cols(Phi + Delta Z_{t,c}) = A + iB, in
// shared memory, then sweeps the upper-triangle 128 x 128 tiles (I <= J) of
//   Re G = A_I^T A_J + B_I^T B_J            (one K = 2*DP contraction)
//   Im G = A_I^T B_J - B_I^T A_J            (two K = DP contractions, the
//                                             second with A negated)
// on the tensor cores with fp32 accumulators in tensor memory, and reduces
// max_{j<k} |G_jk|^2 in the epilogue; the N x N Gram never leaves the SM
// (coherence: arXiv 2207.06374, Sec. "Introduction"; upper triangle only:
// Sec. "Optimization procedure").
//
// Roles (13 warps): warps 0-7 generate column blocks, warps 8-11 (one
// warpgroup) read the accumulators, warp 12 owns tensor memory and issues the
// MMAs.  Shared-memory column blocks and the two accumulator buffers are
// handed over with mbarriers; every wait is bounded in time and gives up by
// setting an error bit instead of spinning forever.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "kernels.h"
#include "philox.cuh"

namespace trstmi {
namespace {

constexpr int kDP = 32;                 // padded d: K = 2*kDP = 64 bf16 = 128 bytes / column
constexpr int kBlockCols = 128;         // columns per block = MMA M = N
constexpr int kBlockBytes = kBlockCols * 2 * kDP * 2;   // 16 KiB
constexpr int kMaxBlocks = 12;          // N <= 1536
constexpr int kGenWarps = 8, kEpiWarps = 8;
constexpr int kEpiWarp0 = kGenWarps;                   // warps 8..15: two whole warpgroups
constexpr int kMmaWarp = kGenWarps + kEpiWarps;        // warp 16
constexpr int kThreads = 32 * (kMmaWarp + 1);          // 544
constexpr uint32_t kTmemCols = 512;                    // 2 buffers x (128 Re + 128 Im)
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
#ifndef TRSTMI_MMA_BACKOFF_NS
#define TRSTMI_MMA_BACKOFF_NS 20
#endif
constexpr unsigned kMmaBackoffNs = TRSTMI_MMA_BACKOFF_NS;  // sleep between MMA-issuer polls

struct ScreenArgs {
  int N, d, nb, ntiles, K;
  uint64_t seed;
  PhiloxKeys keys;  // round keys of the seed, read straight from the parameter bank
  const float2* phi;
  uint32_t c0, t;
  float delta;
  const DevState* st;
  unsigned int* out;
  uint32_t* err;
};

struct SmemCtl {
  unsigned long long blk_full[kMaxBlocks];
  unsigned long long blk_empty[kMaxBlocks];
  unsigned long long acc_full[2];
  unsigned long long acc_empty[2];
  unsigned long long drain;
  uint32_t tmem_base;
  volatile int abort_flag;
  // Decision of a group's elected waiter for one barrier episode, read by the
  // whole group after the named barrier.  Two slots alternate: slot e & 1 is
  // rewritten only after every member has passed barrier e + 1, i.e. after
  // it has read slot e & 1, so all members always act on the same value.
  int gen_go[2], epi_go[2];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  // the thread may sleep in hardware up to the hint (ns) while the phase is
  // pending, so waiting warps do not take issue slots from working ones
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the CTA-wide abort flag and the error bit set) if
// the phase does not complete within kWaitLimitNs or another role aborted.
// Between unsuccessful polls the thread sleeps backoff_ns, so a waiting warp
// leaves the issue slots to the working ones.
__device__ bool mbar_wait(unsigned long long* b, uint32_t parity, SmemCtl* ctl, uint32_t* err,
                          unsigned backoff_ns = 0) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (backoff_ns) __nanosleep(backoff_ns);
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 7u) == 0u) {
      if (ctl->abort_flag) return false;
      if (globaltimer_ns() - t0 > kWaitLimitNs) {
        ctl->abort_flag = 1;
        if (err) atomicOr(err, (uint32_t)kErrTimeout);
        return false;
      }
    }
  }
}

// Hardware named barrier over a role group: blocked warps issue nothing.
__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
constexpr int kBarGen = 1, kBarEpi = 2;

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// UMMA shared-memory descriptor: K-major operand in the 128-byte swizzled
// layout (8 rows x 128 B atoms, 1024 B apart).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1u << 16;                          // leading byte offset (unused: 16 B)
  d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset: 1024 B
  d |= (uint64_t)1u << 46;                          // descriptor version
  d |= (uint64_t)2u << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B both bf16 (format 1)
// or both fp16 (format 0), both K-major, M = N = 128; bit 13 negates A.
template <bool kHalf> struct Idesc {
  static constexpr uint32_t fmt = kHalf ? 0u : 1u;
  static constexpr uint32_t pos = (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 3) << 17) |
                                  ((128u >> 4) << 24);
  static constexpr uint32_t neg_a = pos | (1u << 13);
};

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool kHalf> __device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (kHalf) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  } else {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  }
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Column r (0..127) of a block, 16-byte chunk c (0..7) -> byte offset in the
// block: 8-row atoms of 1024 B, chunk index XOR-swizzled by the row.
__device__ __forceinline__ uint32_t swz_offset(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// One candidate to screen.
struct ScreenItem {
  int N, d, nb, ntiles;
  const float2* phi;
  uint64_t seed;
  uint32_t cand, t;
  float delta;
  unsigned int* out;   // receives its mu^2 (atomic max of non-negative float bits)
};

// Work source: candidates c0 .. c0+K-1 of one instance; the Philox round keys
// come from the kernel parameters, which the instructions read directly.
struct OneInstance {
  ScreenArgs a;
  __device__ bool launch(uint32_t& t, float& delta) const {
    t = a.t;
    delta = a.delta;
    if (a.st) {
      if (!a.st->active || !a.st->use_screen) return false;
      t = a.st->t + 1u;
      delta = (float)a.st->delta_used;
    }
    return true;
  }
  __device__ int count() const { return a.K; }
  __device__ bool item(int idx, uint32_t t, float delta, ScreenItem& it) const {
    it.N = a.N; it.d = a.d; it.nb = a.nb; it.ntiles = a.ntiles;
    it.phi = a.phi; it.seed = a.seed;
    it.cand = a.c0 + (uint32_t)idx; it.t = t; it.delta = delta;
    it.out = a.out + idx;
    return true;
  }
  __device__ PhiloxOut philox(uint32_t e, const ScreenItem& it) const {
    return philox4x32_10_keys(e, it.cand, it.t, 0u, a.keys);
  }
  __device__ uint32_t* err() const { return a.err; }
};

// Work source: (instance, candidate) items of many instances; every instance
// brings its own frame, seed, iteration counter and radius (its DevState),
// and is skipped unless it is active and ranks with the screen this
// iteration (all roles read the same, unchanging state, so they agree).
struct ManyInstances {
  const ScreenSlot* slots;
  const uint2* items;
  int n_items;
  uint32_t* error;
  __device__ bool launch(uint32_t&, float&) const { return true; }
  __device__ int count() const { return n_items; }
  __device__ bool item(int idx, uint32_t, float, ScreenItem& it) const {
    const uint2 w = items[idx];
    const ScreenSlot& s = slots[w.x];
    const DevState* st = s.st;
    if (!st->active || !st->use_screen) return false;
    it.N = s.N; it.d = s.d;
    it.nb = (s.N + kBlockCols - 1) / kBlockCols;
    it.ntiles = it.nb * (it.nb + 1) / 2;
    it.phi = s.phi32; it.seed = s.seed;
    it.cand = w.y; it.t = st->t + 1u; it.delta = (float)st->delta_used;
    it.out = s.mu2 + w.y;
    return true;
  }
  __device__ PhiloxOut philox(uint32_t e, const ScreenItem& it) const {
    return philox4x32_10(e, it.cand, it.t, 0u, seed_lo(it.seed), seed_hi(it.seed));
  }
  __device__ uint32_t* err() const { return error; }
};

// 17 warps: one SM sub-partition (16K registers) holds 5 of them, so a
// thread may use at most 16384 / (5 * 32) -> 96 registers
template <bool kHalf, class Src>
__global__ void __maxnreg__(96) k_screen(const Src src) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ SmemCtl ctl;
  // 1024-byte aligned operand area
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* xs = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t xs_addr = smem_u32(xs);

  uint32_t t0;
  float delta0;
  if (!src.launch(t0, delta0)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* err = src.err();
  const int nitems = src.count();

  if (threadIdx.x == 0) {
    for (int b = 0; b < kMaxBlocks; ++b) {
      mbar_init(&ctl.blk_full[b], kGenWarps);
      mbar_init(&ctl.blk_empty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.acc_full[b], 1);
      mbar_init(&ctl.acc_empty[b], kEpiWarps);
    }
    mbar_init(&ctl.drain, 1);
    ctl.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(&ctl.tmem_base)),
        "r"(kTmemCols)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl.tmem_base;

  if (warp < kGenWarps) {
    // ------------------------------------------------------- generators
    const int g = threadIdx.x;            // 0..255
    const int r = g >> 1, h = g & 1;      // column within the block, half of the entries
    // block b has been filled before (bit b of filled) and the parity of its
    // fill count (bit b of fillpar); the named-barrier episode counter
    uint32_t filled = 0u, fillpar = 0u, ep = 0u;
    for (int idx = blockIdx.x; idx < nitems; idx += gridDim.x) {
      ScreenItem it;
      if (!src.item(idx, t0, delta0, it)) continue;
      const int d = it.d, P = (d + 1) >> 1;
      for (int b = 0; b < it.nb; ++b) {
        if ((filled >> b) & 1u) {
          // one thread polls for the previous fill's release; the other
          // generator warps block in hardware
          const int slot = (int)(ep++ & 1u);
          if (g == 0)
            ctl.gen_go[slot] = mbar_wait(&ctl.blk_empty[b], ((fillpar >> b) & 1u) ^ 1u, &ctl, err,
                                         64) ? 1 : 0;
          group_sync(kBarGen, 32 * kGenWarps);
          if (!ctl.gen_go[slot]) goto gen_done;
        }
        const int j = b * kBlockCols + r;
        float xr[16], xi[16];
        float s = 0.f;
        if (j < it.N && d == kDP) {
          // full width: entries 16h .. 16h+15 are 128 contiguous bytes of phi
          const float4* col4 = reinterpret_cast<const float4*>(it.phi + (size_t)j * kDP + 16 * h);
          float4 v[8];
#pragma unroll
          for (int pp = 0; pp < 8; ++pp) v[pp] = __ldg(col4 + pp);
#pragma unroll
          for (int pp = 0; pp < 8; ++pp) {
            const uint32_t p = (uint32_t)(8 * h + pp);
            const PhiloxOut u = src.philox((uint32_t)j * (uint32_t)(kDP / 2) + p, it);
            perturb_fast(u.x[0], u.x[1], it.delta, v[pp].x, v[pp].y, xr[2 * pp], xi[2 * pp]);
            perturb_fast(u.x[2], u.x[3], it.delta, v[pp].z, v[pp].w, xr[2 * pp + 1], xi[2 * pp + 1]);
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) s = fmaf(xr[e], xr[e], fmaf(xi[e], xi[e], s));
        } else if (j < it.N) {
          const float2* col = it.phi + (size_t)j * d;
#pragma unroll
          for (int pp = 0; pp < 8; ++pp) {
            const int p = 8 * h + pp;
            if (p < P) {
              const PhiloxOut u = src.philox((uint32_t)j * (uint32_t)P + (uint32_t)p, it);
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int i = 2 * p + e;
                float vr = 0.f, vi = 0.f;
                if (i < d) {
                  const float2 v = col[i];
                  perturb_fast(u.x[2 * e], u.x[2 * e + 1], it.delta, v.x, v.y, vr, vi);
                }
                xr[2 * pp + e] = vr;
                xi[2 * pp + e] = vi;
                s = fmaf(vr, vr, fmaf(vi, vi, s));
              }
            } else {
              xr[2 * pp] = xr[2 * pp + 1] = 0.f;
              xi[2 * pp] = xi[2 * pp + 1] = 0.f;
            }
          }
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) { xr[e] = 0.f; xi[e] = 0.f; }
        }
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        const float inv = s > 0.f ? rsqrtf(s) : 0.f;
        unsigned char* blk = xs + b * kBlockBytes;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          uint4 re, im;
          const int e0 = 8 * half;
          re.x = pack2<kHalf>(xr[e0 + 0] * inv, xr[e0 + 1] * inv);
          re.y = pack2<kHalf>(xr[e0 + 2] * inv, xr[e0 + 3] * inv);
          re.z = pack2<kHalf>(xr[e0 + 4] * inv, xr[e0 + 5] * inv);
          re.w = pack2<kHalf>(xr[e0 + 6] * inv, xr[e0 + 7] * inv);
          im.x = pack2<kHalf>(xi[e0 + 0] * inv, xi[e0 + 1] * inv);
          im.y = pack2<kHalf>(xi[e0 + 2] * inv, xi[e0 + 3] * inv);
          im.z = pack2<kHalf>(xi[e0 + 4] * inv, xi[e0 + 5] * inv);
          im.w = pack2<kHalf>(xi[e0 + 6] * inv, xi[e0 + 7] * inv);
          // real parts of entries 16h + 8half .. +7 -> chunk 2h + half;
          // imaginary parts -> chunk 4 + 2h + half
          *reinterpret_cast<uint4*>(blk + swz_offset(r, 2 * h + half)) = re;
          *reinterpret_cast<uint4*>(blk + swz_offset(r, 4 + 2 * h + half)) = im;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl.blk_full[b]);
        filled |= 1u << b;
        fillpar ^= 1u << b;
      }
    }
  gen_done:;
  } else if (warp < kMmaWarp) {
    // --------------------------------------------------------- epilogue
    // warps 8..11 take accumulator columns 0..63 of every tile, warps 12..15
    // columns 64..127; within a warpgroup, warp w reads TMEM lanes 32(w%4)..
    const int ew = warp - kEpiWarp0;
    const int qw = ew & 3;                           // TMEM lane quarter
    const int colh = 64 * (ew >> 2);                 // first accumulator column of this warp
    uint32_t gt = 0;                                 // tile counter
    for (int idx = blockIdx.x; idx < nitems; idx += gridDim.x) {
      ScreenItem it;
      if (!src.item(idx, t0, delta0, it)) continue;
      const int nb = it.nb;
      // four independent running maxima keep the max chain off the critical path
      float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
      bool ok = true;
      // tiles in the MMA issuer's row-major order: I = 0..nb-1, J = I..nb-1
      int I = 0, J = 0;
      for (int tau = 0; tau < it.ntiles; ++tau, ++gt, J = (J + 1 < nb) ? J + 1 : ++I) {
        const uint32_t buf = gt & 1u, use = gt >> 1;
        // one thread polls; the other epilogue warps block in hardware
        if (ew == 0 && lane == 0)
          ctl.epi_go[gt & 1u] = mbar_wait(&ctl.acc_full[buf], use & 1u, &ctl, err, 32) ? 1 : 0;
        group_sync(kBarEpi, 32 * kEpiWarps);
        if (!ctl.epi_go[gt & 1u]) { ok = false; break; }
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(32 * qw) << 16) + buf * 256u + (uint32_t)colh;
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
          // On a diagonal tile only k > j counts: this warp's rows are
          // 32qw..32qw+31 and the chunk's columns n0..n0+31, so the chunk is
          // entirely below the diagonal (skip), entirely above (no mask) or
          // straddles it (n0 == 32qw: mask column e against row lane).
          const int n0 = colh + 32 * ch;
          const bool diag = (I == J);
          if (diag && n0 < 32 * qw) continue;
          uint32_t re[32], im[32];
          tmem_ld32(base + 32u * ch, re);
          tmem_ld32(base + 128u + 32u * ch, im);
          tmem_ld_wait();
          if (!diag || n0 > 32 * qw) {
            // two pairs per packed multiply / fma, one three-input max
#pragma unroll
            for (int e = 0; e < 32; e += 8) {
              float2 x, y, v;
              x = make_float2(__uint_as_float(re[e]), __uint_as_float(re[e + 1]));
              y = make_float2(__uint_as_float(im[e]), __uint_as_float(im[e + 1]));
              v = __ffma2_rn(y, y, __fmul2_rn(x, x));
              m0 = fmax3(m0, v.x, v.y);
              x = make_float2(__uint_as_float(re[e + 2]), __uint_as_float(re[e + 3]));
              y = make_float2(__uint_as_float(im[e + 2]), __uint_as_float(im[e + 3]));
              v = __ffma2_rn(y, y, __fmul2_rn(x, x));
              m1 = fmax3(m1, v.x, v.y);
              x = make_float2(__uint_as_float(re[e + 4]), __uint_as_float(re[e + 5]));
              y = make_float2(__uint_as_float(im[e + 4]), __uint_as_float(im[e + 5]));
              v = __ffma2_rn(y, y, __fmul2_rn(x, x));
              m2 = fmax3(m2, v.x, v.y);
              x = make_float2(__uint_as_float(re[e + 6]), __uint_as_float(re[e + 7]));
              y = make_float2(__uint_as_float(im[e + 6]), __uint_as_float(im[e + 7]));
              v = __ffma2_rn(y, y, __fmul2_rn(x, x));
              m3 = fmax3(m3, v.x, v.y);
            }
          } else {
            // straddling chunk: column n0 + e against row 32qw + lane
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const float x = __uint_as_float(re[e]), y = __uint_as_float(im[e]);
              const float v = fmaf(x, x, y * y);
              m0 = (e > lane) ? fmaxf(m0, v) : m0;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl.acc_empty[buf]);
      }
      if (!ok) break;
      float m = fmaxf(fmaxf(m0, m1), fmaxf(m2, m3));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) atomicMax(it.out, __float_as_uint(m));
    }
  } else {
    // ------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t gt = 0;
      uint32_t usepar = 0u;   // parity of the next fill of block b to consume (bit b)
      bool ok = true;
      // Row-major sweep: block I is last read in row I (as A for J >= I, as B
      // in rows I' <= I), so it is released right after its row and the next
      // candidate's block I is generated while rows I+1.. still run.  Row 0
      // reads every block; it waits for each one as it first needs it.
      for (int idx = blockIdx.x; idx < nitems && ok; idx += gridDim.x) {
        ScreenItem it;
        if (!src.item(idx, t0, delta0, it)) continue;
        const int nb = it.nb;
        for (int I = 0; I < nb && ok; ++I) {
          for (int J = I; J < nb; ++J, ++gt) {
            if (I == 0) {
              ok = mbar_wait(&ctl.blk_full[J], (usepar >> J) & 1u, &ctl, err, kMmaBackoffNs);
              if (!ok) break;
              usepar ^= 1u << J;
            }
            const uint32_t buf = gt & 1u, use = gt >> 1;
            if (use > 0) {
              ok = mbar_wait(&ctl.acc_empty[buf], (use - 1u) & 1u, &ctl, err, kMmaBackoffNs);
              if (!ok) break;
            }
            tc_fence_after();
            const uint32_t aI = xs_addr + (uint32_t)(I * kBlockBytes);
            const uint32_t bJ = xs_addr + (uint32_t)(J * kBlockBytes);
            const uint32_t dre = tmem + buf * 256u, dim = dre + 128u;
            // Re: sum over the whole K = 2*DP (4 steps of 16)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(dre, smem_desc_sw128(aI + 32u * kk), smem_desc_sw128(bJ + 32u * kk),
                       Idesc<kHalf>::pos, kk > 0 ? 1u : 0u);
            // Im: A_I^T B_J (K slices 0,1 against 2,3) - B_I^T A_J (2,3 against 0,1)
            mma_bf16(dim, smem_desc_sw128(aI + 0u), smem_desc_sw128(bJ + 64u), Idesc<kHalf>::pos, 0u);
            mma_bf16(dim, smem_desc_sw128(aI + 32u), smem_desc_sw128(bJ + 96u), Idesc<kHalf>::pos, 1u);
            mma_bf16(dim, smem_desc_sw128(aI + 64u), smem_desc_sw128(bJ + 0u), Idesc<kHalf>::neg_a, 1u);
            mma_bf16(dim, smem_desc_sw128(aI + 96u), smem_desc_sw128(bJ + 32u), Idesc<kHalf>::neg_a, 1u);
            mma_commit(&ctl.acc_full[buf]);
          }
          if (ok) mma_commit(&ctl.blk_empty[I]);   // row I done: block I is free
        }
      }
      // all issued MMAs complete before tensor memory is released
      mma_commit(&ctl.drain);
      mbar_wait(&ctl.drain, 0u, &ctl, err);
    }
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

size_t screen_smem_bytes(int nb) { return (size_t)nb * kBlockBytes + 1024; }

template <class K> cudaError_t allow_screen_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              std::min((int)screen_smem_bytes(kMaxBlocks),
                                       optin - (int)fa.sharedSizeBytes));
}

// refuse (without launching) a configuration the SM cannot hold
template <class K> cudaError_t screen_fits(K kernel) {
  int fit = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, kThreads,
                                                                screen_smem_bytes(kMaxBlocks));
  if (e != cudaSuccess) return e;
  return fit < 1 ? cudaErrorLaunchOutOfResources : cudaSuccess;
}

}  // namespace

bool screen_supported(int N, int d) {
  const int nb = (N + kBlockCols - 1) / kBlockCols;
  return N >= 2 && d >= 1 && d <= kDP && nb <= kMaxBlocks;
}

cudaError_t init_screen_attributes(int optin) {
  cudaError_t e;
  if ((e = allow_screen_smem(k_screen<false, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<true, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<false, ManyInstances>, optin)) != cudaSuccess) return e;
  return allow_screen_smem(k_screen<true, ManyInstances>, optin);
}

cudaError_t launch_screen(bool fp16, int N, int d, uint64_t seed, const float2* phi32, int K,
                          uint32_t c0, uint32_t t, double delta, const DevState* st,
                          unsigned int* mu2_out, uint32_t* err_flag, int num_sms,
                          cudaStream_t s) {
  if (!screen_supported(N, d) || K < 1) return cudaErrorInvalidValue;
  OneInstance src;
  ScreenArgs& a = src.a;
  a.N = N; a.d = d;
  a.nb = (N + kBlockCols - 1) / kBlockCols;
  a.ntiles = a.nb * (a.nb + 1) / 2;
  a.K = K; a.seed = seed; a.phi = phi32; a.c0 = c0; a.t = t; a.delta = (float)delta;
  a.keys = philox_round_keys(seed);
  a.st = st; a.out = mu2_out; a.err = err_flag;
  const int grid = std::min(K, num_sms);
  cudaError_t e = fp16 ? screen_fits(k_screen<true, OneInstance>)
                       : screen_fits(k_screen<false, OneInstance>);
  if (e != cudaSuccess) return e;
  // the operand area is always reserved for the largest block count, so every
  // descriptor address lies inside the CTA's shared memory
  if (fp16) k_screen<true, OneInstance><<<grid, kThreads, screen_smem_bytes(kMaxBlocks), s>>>(src);
  else k_screen<false, OneInstance><<<grid, kThreads, screen_smem_bytes(kMaxBlocks), s>>>(src);
  return cudaGetLastError();
}

cudaError_t launch_screen_batched(bool fp16, const ScreenSlot* slots, const uint2* items,
                                  int n_items, uint32_t* err_flag, int num_sms, cudaStream_t s) {
  if (n_items < 1) return cudaSuccess;
  ManyInstances src;
  src.slots = slots;
  src.items = items;
  src.n_items = n_items;
  src.error = err_flag;
  const int grid = std::min(n_items, num_sms);
  cudaError_t e = fp16 ? screen_fits(k_screen<true, ManyInstances>)
                       : screen_fits(k_screen<false, ManyInstances>);
  if (e != cudaSuccess) return e;
  if (fp16) k_screen<true, ManyInstances><<<grid, kThreads, screen_smem_bytes(kMaxBlocks), s>>>(src);
  else k_screen<false, ManyInstances><<<grid, kThreads, screen_smem_bytes(kMaxBlocks), s>>>(src);
  return cudaGetLastError();
}

}  // namespace trstmi
