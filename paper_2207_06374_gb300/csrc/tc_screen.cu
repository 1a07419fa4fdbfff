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
// Roles (20 warps): ten generator warps fill column blocks into a ring of
// shared-memory slots, eight epilogue warps read the accumulators, warp 0
// owns tensor memory and issues the MMAs.  Slots and
// the two accumulator buffers are handed over with mbarriers; every wait is
// bounded in time and gives up by setting an error bit instead of spinning
// forever.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "kernels.h"
#include "philox.cuh"
#include "tile.cuh"

namespace trstmi {
namespace {

constexpr int kBlockCols = 128;         // columns per block = MMA M = N
// Operand formats (ScreenFmt): a column block is 128 columns x 2 DP values,
// DP the padded d.
// bf16 / fp16 (d <= 32, DP = 32): one 128-byte swizzle atom per column (Re
// 0..31 then Im 0..31), 16 KiB per block, twelve slots (N <= 1536).
// tf32 (d <= 32, DP = 32) and wide bf16 / fp16 (d <= 64, DP = 64): two atoms
// per column, Re in the first 16 KiB of the block and Im in the second (32
// tf32 or 64 bf16 values = 128 bytes each), 32 KiB per block, six slots
// (N <= 768).  Either way the slots fill the same 192 KiB.
template <int F> struct FmtTraits {
  static constexpr bool kWide16 = F == kScreenBF16W || F == kScreenFP16W;
  static constexpr bool kTwoAtoms = F == kScreenTF32 || kWide16;
  static constexpr int kDP = kWide16 ? 64 : 32;
  static constexpr int kEntries = kDP / 4;        // entries of a column per generator lane
  static constexpr int kBlockBytes = kTwoAtoms ? 32768 : 16384;
  static constexpr int kSlots = kTwoAtoms ? 6 : 12;
  // instruction-descriptor operand format: fp16 0, bf16 1 (kind::f16), tf32 2 (kind::tf32)
  static constexpr uint32_t kAB = (F == kScreenFP16 || F == kScreenFP16W) ? 0u
                                  : (F == kScreenBF16 || F == kScreenBF16W) ? 1u : 2u;
};
constexpr int kOperandBytes = 12 * 16384;
constexpr int kRing = 12;               // barrier slots: the largest ring
// Warp roles.  A warp runs on SM sub-partition (warp % 4), and reads only
// the tensor-memory lanes 32 (warp % 4) .. +31.  Sub-partition 0 holds the two
// MMA issuers (warps 0 and 16), two epilogue warps (4 and 8) and a single
// generator (12), so the long integer-multiply streams of the random draws
// rarely delay an MMA issue; the other nine generators (warps 1-3, 13-15,
// 17-19) share sub-partitions 1-3 with the other epilogue warps.
// Each issuer owns one accumulator buffer and issues every other tile: an
// MMA instruction holds its issuing thread for about as long as the tensor
// core takes to run it at N = 128, and a tile's hand-off (commit, epilogue,
// release) takes longer than a tile's MMAs, so with one issuer the tensor
// core idles while that thread waits for a buffer; with two, one issuer's
// tile runs while the other waits.
constexpr int kWarps = 20;
constexpr int kThreads = 32 * kWarps;                  // 640
constexpr int kMmaWarp = 0, kMmaWarp2 = 16;
constexpr int kEpiWarp0 = 4, kEpiWarps = 8;            // warps 4..11: two warpgroups
constexpr int kGenWarps = 10;
constexpr int kOctets = 16;                            // 8-column units of a block
__host__ __device__ constexpr int gen_index(int w) {
  return w == 12 ? 9
         : (w % 4 == 0 || (w >= kEpiWarp0 && w < kEpiWarp0 + kEpiWarps)) ? -1
         : w < 4 ? w - 1 : w < 16 ? w - 13 + 3 : w - 17 + 6;
}
static_assert(gen_index(1) == 0 && gen_index(15) == 5 && gen_index(19) == 8 &&
                  gen_index(12) == kGenWarps - 1 && gen_index(16) == -1 && gen_index(0) == -1,
              "roles");
constexpr uint32_t kTmemCols = 512;                    // 2 buffers x (128 Re + 128 Im)
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // default bound of every wait
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
  unsigned long long wait_limit_ns;   // bound of every mbarrier wait
  int withhold_blocks;                // test of the bounded waits: generators fill nothing
};

struct SmemCtl {
  unsigned long long blk_full[kRing];    // slot filled (8 generator warps arrive)
  unsigned long long blk_empty[kRing];   // slot's last MMA done (tcgen05.commit)
  unsigned long long acc_full[2];        // accumulator buffer ready (tcgen05.commit)
  unsigned long long acc_empty[2];       // buffer read (the 8 epilogue warps)
  unsigned long long drain;
  uint32_t tmem_base;
  volatile int abort_flag;
  unsigned long long wait_limit_ns;
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

// The next phase of b completes when `bytes` more have landed (and one arrival).
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on b's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
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
// the phase does not complete within ctl->wait_limit_ns or another role aborted.
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
      if (globaltimer_ns() - t0 > ctl->wait_limit_ns) {
        ctl->abort_flag = 1;
        if (err) atomicOr(err, (uint32_t)kErrTimeout);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// UMMA shared-memory descriptor of a K-major operand in the 128-byte
// swizzled layout (8 rows x 128 B atoms, 1024 B apart): start address >> 4 in
// bits 0-13, leading byte offset 1 (unused) in bits 16-29, stride byte offset
// 1024 >> 4 in bits 32-45, version 1 in bits 46-47, swizzle mode 2 in bits
// 61-63.  A step of 16 bf16 along K is 32 bytes, i.e. +2 in the low word.
// Instruction descriptor: D fp32, A and B of the same format (fp16 0 or
// bf16 1 with kind::f16, tf32 2 with kind::tf32), both K-major,
// M = N = 128; bit 13 negates A.
template <int F> struct Idesc {
  static constexpr uint32_t fmt = FmtTraits<F>::kAB;
  static constexpr uint32_t pos = (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 3) << 17) |
                                  ((128u >> 4) << 24);
  static constexpr uint32_t neg_a = pos | (1u << 13);
};

// High word of every operand descriptor (stride byte offset 1024 B, version
// bit, 128-byte swizzle); the low word carries the start address.
constexpr uint32_t kDescHi = (1024u >> 4) | (1u << 14) | (2u << 29);
__device__ __forceinline__ uint32_t desc_lo(uint32_t addr) {
  return ((addr >> 4) & 0x3FFFu) | (1u << 16);
}

// One MMA from the low descriptor words (the high word is kDescHi).
template <int F>
__device__ __forceinline__ void mma_lo(uint32_t tmem_d, uint32_t alo, uint32_t blo,
                                       uint32_t idesc, uint32_t accumulate, uint32_t hi) {
  if constexpr (F == kScreenTF32) {
    asm volatile(
        "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %4, 0;\n"
        " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %5};\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(alo), "r"(blo), "r"(idesc), "r"(accumulate), "r"(hi)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %4, 0;\n"
        " mov.b64 da, {%1, %5};\n mov.b64 db, {%2, %5};\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(alo), "r"(blo), "r"(idesc), "r"(accumulate), "r"(hi)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// fp32 value rounded to tf32 (nearest, ties away), as the 32-bit word the MMA reads
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int F> __device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (FmtTraits<F>::kAB == 0u) {
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

// Where the column blocks of one item live.  The upper-triangle tiles are
// swept band by band: a band is Rb <= R consecutive blocks r0 .. r0+Rb-1,
// resident while its own triangle is swept row by row, and, when blocks lie
// to its right (r0+Rb .. nb-1), while those stream through two further slots,
// each used for one column of Rb tiles.  An item whose blocks all fit
// (nb <= kSlots) is one band without a stream and releases its blocks row by
// row, so the next item's first blocks fill the slots freed early.  Band
// blocks go round a ring of B slots, stream blocks round the last two; bit s
// of `par` is the parity of slot s's next fill, bit s of `used` records that
// it was filled before.  Generators and the MMA issuer walk the same block
// sequence (per band: its blocks, then its stream blocks) and so derive the
// same slots and parities; a slot is always released before its next fill is
// needed, because blocks are released in the order they are first used.
template <int F> struct SlotPlan {
  static constexpr int kS = FmtTraits<F>::kSlots;
  static constexpr int kStream = 2;
  // the state is packed so that it costs the generators' hot loop few
  // registers: pu = par | used << 16; ring = bp | sp << 8 | B << 16 | R << 24;
  // band = b0 | Rb << 8; bsnap = par | used << 16 as the band began
  uint32_t pu = 0, ring = 0, band = 0, bsnap = 0;
  int nb = 0, r0 = 0;
  __device__ __forceinline__ int R() const { return (int)(ring >> 24); }
  __device__ __forceinline__ int B() const { return (int)((ring >> 16) & 0xffu); }
  __device__ __forceinline__ int Rb() const { return (int)(band >> 8); }
  __device__ __forceinline__ void begin_item(int nb_) {
    nb = nb_;
    const bool fits = nb <= kS;
    const uint32_t R_ = (uint32_t)(fits ? nb : kS - kStream), B_ = (uint32_t)(fits ? kS : kS - kStream);
    uint32_t bp = ring & 0xffu;
    if (bp >= B_) bp = 0;
    ring = bp | (ring & 0xff00u) | (B_ << 16) | (min(R_, 255u) << 24);
  }
  __device__ __forceinline__ void begin_band(int r0_) {
    r0 = r0_;
    const int Rb_ = min(R(), nb - r0);
    const uint32_t bp = ring & 0xffu;
    band = bp | ((uint32_t)Rb_ << 8);
    bsnap = pu;
    for (int q = 0; q < Rb_; ++q) {
      const uint32_t m = 1u << slot_band(q);
      pu = (pu ^ m) | (m << 16);
    }
    ring = (ring & ~0xffu) | (uint32_t)((bp + Rb_) % B());
  }
  __device__ __forceinline__ bool streams() const { return r0 + Rb() < nb; }
  __device__ __forceinline__ int slot_band(int q) const {
    const int s = (int)(band & 0xffu) + q;
    return s >= B() ? s - B() : s;
  }
  __device__ __forceinline__ uint32_t parity_band(int q) const { return (bsnap >> slot_band(q)) & 1u; }
  __device__ __forceinline__ bool used_band(int q) const {
    return ((bsnap >> (16 + slot_band(q))) & 1u) != 0;
  }
  // the next stream block's slot, the parity of this fill and whether the
  // slot was filled before
  __device__ __forceinline__ int next_stream(uint32_t& p, bool& u) {
    const uint32_t sp = (ring >> 8) & 1u;
    const int s = kS - kStream + (int)sp;
    ring ^= 1u << 8;
    p = (pu >> s) & 1u;
    u = ((pu >> (16 + s)) & 1u) != 0;
    pu = (pu ^ (1u << s)) | (1u << (16 + s));
    return s;
  }
};

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
  __device__ PhiloxCand cand(const ScreenItem& it) const {
    return philox_cand(it.cand, it.t, a.keys.k0[0], a.keys.k0[1], a.keys.k1[1]);
  }
  __device__ PhiloxOut philox(uint32_t e, const PhiloxCand& pc, const ScreenItem&) const {
    const PhiloxKeys& k = a.keys;
    return philox_from_cand(e, pc, k.k1[0], [&](int r, uint32_t& k0, uint32_t& k1) {
      k0 = k.k0[r];
      k1 = k.k1[r];
    });
  }
  __device__ uint32_t* err() const { return a.err; }
  __device__ unsigned long long wait_limit() const { return a.wait_limit_ns; }
  __device__ bool withhold() const { return a.withhold_blocks != 0; }
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
  __device__ PhiloxCand cand(const ScreenItem& it) const {
    const uint32_t lo = seed_lo(it.seed), hi = seed_hi(it.seed);
    return philox_cand(it.cand, it.t, lo, lo + 0x9E3779B9u, hi + 0xBB67AE85u);
  }
  __device__ PhiloxOut philox(uint32_t e, const PhiloxCand& pc, const ScreenItem& it) const {
    const uint32_t lo = seed_lo(it.seed), hi = seed_hi(it.seed);
    return philox_from_cand(e, pc, hi, [&](int r, uint32_t& k0, uint32_t& k1) {
      k0 = lo + (uint32_t)r * 0x9E3779B9u;
      k1 = hi + (uint32_t)r * 0xBB67AE85u;
    });
  }
  __device__ uint32_t* err() const { return error; }
  __device__ unsigned long long wait_limit() const { return kWaitLimitNs; }
  __device__ bool withhold() const { return false; }
};

// Bounded wait by every lane of a warp; the warp acts on the unanimous result.
__device__ __forceinline__ bool warp_wait(unsigned long long* b, uint32_t parity, SmemCtl* ctl,
                                          uint32_t* err, unsigned backoff_ns) {
  const bool ok = mbar_wait(b, parity, ctl, err, backoff_ns);
  return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
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

// Waits for the thread's outstanding tensor-memory loads.  The destination
// registers of the awaited loads are passed through, so no use of them can be
// placed before the wait.
template <int W>
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&a)[W], uint32_t (&b)[W]);

template <>
__device__ __forceinline__ void tmem_wait_ld<16>(uint32_t (&a)[16], uint32_t (&b)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                 "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]),
                 "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]),
                 "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                 "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]),
                 "+r"(b[14]), "+r"(b[15])
               :
               : "memory");
}

template <>
__device__ __forceinline__ void tmem_wait_ld<32>(uint32_t (&a)[32], uint32_t (&b)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                 "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]),
                 "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]), "+r"(a[16]), "+r"(a[17]),
                 "+r"(a[18]), "+r"(a[19]), "+r"(a[20]), "+r"(a[21]), "+r"(a[22]), "+r"(a[23]),
                 "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]), "+r"(a[28]), "+r"(a[29]),
                 "+r"(a[30]), "+r"(a[31]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                 "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]),
                 "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]),
                 "+r"(b[16]), "+r"(b[17]), "+r"(b[18]), "+r"(b[19]), "+r"(b[20]), "+r"(b[21]),
                 "+r"(b[22]), "+r"(b[23]), "+r"(b[24]), "+r"(b[25]), "+r"(b[26]), "+r"(b[27]),
                 "+r"(b[28]), "+r"(b[29]), "+r"(b[30]), "+r"(b[31])
               :
               : "memory");
}

// max of |G|^2 over W accumulator columns (Re in re, Im in im): two pairs per
// packed multiply / fma, one three-input max per two pairs, spread over
// eight running maxima so no max chain sits on the critical path.
template <int W>
__device__ __forceinline__ void absmax(const uint32_t (&re)[W], const uint32_t (&im)[W],
                                       float (&m)[8]) {
#pragma unroll
  for (int e = 0; e < W; e += 2) {
    const float2 x = make_float2(__uint_as_float(re[e]), __uint_as_float(re[e + 1]));
    const float2 y = make_float2(__uint_as_float(im[e]), __uint_as_float(im[e + 1]));
    const float2 v = __ffma2_rn(y, y, __fmul2_rn(x, x));
    m[(e >> 1) & 7] = fmax3(m[(e >> 1) & 7], v.x, v.y);
  }
}

// The MMAs of one tile: A (block I) at descriptor low word alo, B (block J)
// at blo, into the Re accumulator at tensor-memory column dre and the Im one
// at dim (the high descriptor word is hi).
template <int F>
__device__ __forceinline__ void issue_tile_mmas(uint32_t alo, uint32_t blo, uint32_t dre,
                                                uint32_t dim, uint32_t hi) {
  if constexpr (FmtTraits<F>::kTwoAtoms) {
    // K steps of 8 tf32 or 16 bf16 / fp16 = 32 bytes = +2 in the low
    // word; the second atom (Im parts) is 16 KiB = +1024 further
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)   // Re: A_I^T A_J ...
      mma_lo<F>(dre, alo + 2u * kk, blo + 2u * kk, Idesc<F>::pos, kk > 0 ? 1u : 0u, hi);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)   // ... + B_I^T B_J
      mma_lo<F>(dre, alo + 1024u + 2u * kk, blo + 1024u + 2u * kk, Idesc<F>::pos, 1u, hi);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)   // Im: A_I^T B_J ...
      mma_lo<F>(dim, alo + 2u * kk, blo + 1024u + 2u * kk, Idesc<F>::pos, kk > 0 ? 1u : 0u, hi);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)   // ... - B_I^T A_J
      mma_lo<F>(dim, alo + 1024u + 2u * kk, blo + 2u * kk, Idesc<F>::neg_a, 1u, hi);
  } else {
    // Re: sum over the whole K = 2*DP (4 steps of 16 = +2 in the low word)
    mma_lo<F>(dre, alo + 0u, blo + 0u, Idesc<F>::pos, 0u, hi);
    mma_lo<F>(dre, alo + 2u, blo + 2u, Idesc<F>::pos, 1u, hi);
    mma_lo<F>(dre, alo + 4u, blo + 4u, Idesc<F>::pos, 1u, hi);
    mma_lo<F>(dre, alo + 6u, blo + 6u, Idesc<F>::pos, 1u, hi);
    // Im: A_I^T B_J (K slices 0,1 against 2,3) - B_I^T A_J (2,3 against 0,1)
    mma_lo<F>(dim, alo + 0u, blo + 4u, Idesc<F>::pos, 0u, hi);
    mma_lo<F>(dim, alo + 2u, blo + 6u, Idesc<F>::pos, 1u, hi);
    mma_lo<F>(dim, alo + 4u, blo + 0u, Idesc<F>::neg_a, 1u, hi);
    mma_lo<F>(dim, alo + 6u, blo + 2u, Idesc<F>::neg_a, 1u, hi);
  }
}

// Octet o (columns 8o .. 8o+7) of column block jb of candidate `it` into the
// block at blk, in the operand layout of format F: lane l takes column
// 8o + (l & 7) and the quarter l >> 3 of its DP padded entries (E = DP/4 of
// them, E/2 draws), draws and perturbs them, normalises the column (the
// quarter sums joined by two shuffles) and stores its chunks; the eight lanes
// of one quarter write eight different 16-byte chunks of a swizzled row
// group, so the stores are free of bank conflicts.
template <int F, class Src>
__device__ __forceinline__ void gen_octet(const Src& src, const ScreenItem& it,
                                          const PhiloxCand& pc, int o, int jb,
                                          unsigned char* blk, int lane) {
  constexpr int kDP = FmtTraits<F>::kDP, kE = FmtTraits<F>::kEntries;
  const int q = lane >> 3;
  const int d = it.d, P = (d + 1) >> 1;
  const int r = 8 * o + (lane & 7);        // row of the block (column of Phi)
  const int j = jb * kBlockCols + r;
  float2 x[kE];
  float2 ss = make_float2(0.f, 0.f);
  if (j < it.N && d == kDP) {
    // full width: entries Eq .. Eq+E-1 are 8E contiguous bytes of phi,
    // read as float4 (two entries) in groups of eight entries
#pragma unroll
    for (int h = 0; h < kE / 8; ++h) {
      const float4* col4 =
          reinterpret_cast<const float4*>(it.phi + (size_t)j * kDP + kE * q + 8 * h);
      float4 v[4];
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) v[pp] = __ldg(col4 + pp);
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) {
        const PhiloxOut w = src.philox(
            (uint32_t)j * (uint32_t)(kDP / 2) + (uint32_t)(kE / 2 * q + 4 * h + pp), pc, it);
        perturb2_fast(w.x, it.delta, make_float2(v[pp].x, v[pp].y),
                      make_float2(v[pp].z, v[pp].w), x[8 * h + 2 * pp],
                      x[8 * h + 2 * pp + 1]);
      }
    }
  } else if (j < it.N) {
    const float2* col = it.phi + (size_t)j * d;
#pragma unroll
    for (int pp = 0; pp < kE / 2; ++pp) {
      const int p = kE / 2 * q + pp;
      x[2 * pp] = x[2 * pp + 1] = make_float2(0.f, 0.f);
      if (p < P) {
        const PhiloxOut w = src.philox((uint32_t)j * (uint32_t)P + (uint32_t)p, pc, it);
        const int i = 2 * p;
        const float2 v0 = col[i];
        const float2 v1 = (i + 1 < d) ? col[i + 1] : make_float2(0.f, 0.f);
        float2 y0, y1;
        perturb2_fast(w.x, it.delta, v0, v1, y0, y1);
        x[2 * pp] = y0;
        if (i + 1 < d) x[2 * pp + 1] = y1;
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < kE; ++e) x[e] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int e = 0; e < kE; ++e) ss = __ffma2_rn(x[e], x[e], ss);
  float sn = ss.x + ss.y;
  sn += __shfl_xor_sync(0xffffffffu, sn, 8);
  sn += __shfl_xor_sync(0xffffffffu, sn, 16);
  const float inv = sn > 0.f ? rsqrtf(sn) : 0.f;
  const float2 inv2 = make_float2(inv, inv);
#pragma unroll
  for (int e = 0; e < kE; ++e) x[e] = __fmul2_rn(x[e], inv2);
  if constexpr (FmtTraits<F>::kWide16) {
    // real parts of entries 16q .. 16q+15 -> chunks 2q, 2q+1 of the
    // first atom; imaginary parts -> the same chunks of the second
    uint4 re0, re1, im0, im1;
    re0.x = pack2<F>(x[0].x, x[1].x);   re1.x = pack2<F>(x[8].x, x[9].x);
    re0.y = pack2<F>(x[2].x, x[3].x);   re1.y = pack2<F>(x[10].x, x[11].x);
    re0.z = pack2<F>(x[4].x, x[5].x);   re1.z = pack2<F>(x[12].x, x[13].x);
    re0.w = pack2<F>(x[6].x, x[7].x);   re1.w = pack2<F>(x[14].x, x[15].x);
    im0.x = pack2<F>(x[0].y, x[1].y);   im1.x = pack2<F>(x[8].y, x[9].y);
    im0.y = pack2<F>(x[2].y, x[3].y);   im1.y = pack2<F>(x[10].y, x[11].y);
    im0.z = pack2<F>(x[4].y, x[5].y);   im1.z = pack2<F>(x[12].y, x[13].y);
    im0.w = pack2<F>(x[6].y, x[7].y);   im1.w = pack2<F>(x[14].y, x[15].y);
    *reinterpret_cast<uint4*>(blk + swz_offset(r, 2 * q)) = re0;
    *reinterpret_cast<uint4*>(blk + swz_offset(r, 2 * q + 1)) = re1;
    *reinterpret_cast<uint4*>(blk + 16384 + swz_offset(r, 2 * q)) = im0;
    *reinterpret_cast<uint4*>(blk + 16384 + swz_offset(r, 2 * q + 1)) = im1;
  } else if constexpr (F == kScreenTF32) {
    // real parts of entries 8q .. 8q+7 -> chunks 2q, 2q+1 of the first
    // atom; imaginary parts -> the same chunks of the second
    const uint4 cr0 = make_uint4(to_tf32(x[0].x), to_tf32(x[1].x), to_tf32(x[2].x), to_tf32(x[3].x));
    const uint4 cr1 = make_uint4(to_tf32(x[4].x), to_tf32(x[5].x), to_tf32(x[6].x), to_tf32(x[7].x));
    const uint4 ci0 = make_uint4(to_tf32(x[0].y), to_tf32(x[1].y), to_tf32(x[2].y), to_tf32(x[3].y));
    const uint4 ci1 = make_uint4(to_tf32(x[4].y), to_tf32(x[5].y), to_tf32(x[6].y), to_tf32(x[7].y));
    *reinterpret_cast<uint4*>(blk + swz_offset(r, 2 * q)) = cr0;
    *reinterpret_cast<uint4*>(blk + swz_offset(r, 2 * q + 1)) = cr1;
    *reinterpret_cast<uint4*>(blk + 16384 + swz_offset(r, 2 * q)) = ci0;
    *reinterpret_cast<uint4*>(blk + 16384 + swz_offset(r, 2 * q + 1)) = ci1;
  } else {
    uint4 re, im;
    re.x = pack2<F>(x[0].x, x[1].x);
    re.y = pack2<F>(x[2].x, x[3].x);
    re.z = pack2<F>(x[4].x, x[5].x);
    re.w = pack2<F>(x[6].x, x[7].x);
    im.x = pack2<F>(x[0].y, x[1].y);
    im.y = pack2<F>(x[2].y, x[3].y);
    im.z = pack2<F>(x[4].y, x[5].y);
    im.w = pack2<F>(x[6].y, x[7].y);
    // real parts of entries 8q .. 8q+7 -> chunk q; imaginary -> chunk 4 + q
    *reinterpret_cast<uint4*>(blk + swz_offset(r, q)) = re;
    *reinterpret_cast<uint4*>(blk + swz_offset(r, 4 + q)) = im;
  }
}

// 20 warps: one SM sub-partition (16K registers) holds 5 of them, so a
// thread may use at most 16384 / (5 * 32) -> 96 registers
template <int F, class Src>
__global__ void __maxnreg__(96) k_screen(const Src src) {
  constexpr int kBlockBytes = FmtTraits<F>::kBlockBytes;
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
    for (int b = 0; b < kRing; ++b) {
      mbar_init(&ctl.blk_full[b], kOctets);
      mbar_init(&ctl.blk_empty[b], 2);   // both MMA issuers commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl.acc_full[b], 1);
      mbar_init(&ctl.acc_empty[b], kEpiWarps);
    }
    mbar_init(&ctl.drain, 2);
    ctl.abort_flag = 0;
    ctl.wait_limit_ns = src.wait_limit();
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

  const int gi = gen_index(warp);
  if (gi >= 0) {
    // ------------------------------------------------------- generators
    // The column blocks of successive candidates go round a ring of kRing
    // slots (global block number gb -> slot gb % kRing, fill gb / kRing), so
    // the next candidate's first blocks are generated into free slots while
    // the current one is still being swept.  The work is cut into 8-column
    // units (octets), numbered consecutively over all blocks of this CTA;
    // generator gi takes the units u = gi (mod kGenWarps).  In a unit, lane l
    // takes column 8o + (l & 7) and the quarter q = l >> 3 of its DP padded
    // entries: E = DP/4 of them (Eq .. Eq+E-1, E/2 draws); the eight lanes of
    // one quarter write eight different 16-byte chunks of a swizzled row
    // group, so the stores are free of bank conflicts.  Each unit's warp
    // arrives once on the slot's fill barrier (kOctets arrivals complete a
    // fill).  The lanes' layout within a unit is gen_octet's.
    SlotPlan<F> plan;
    uint32_t ucount = 0;      // octet units so far (16 per block instance)
    const int gen_items = src.withhold() ? 0 : nitems;
    for (int idx = blockIdx.x; idx < gen_items; idx += gridDim.x) {
      ScreenItem it;
      if (!src.item(idx, t0, delta0, it)) continue;
      const PhiloxCand pc = src.cand(it);
      // octet o of column block jb into slot `slot`
      auto fill_octet = [&](int o, int jb, int slot) {
        gen_octet<F>(src, it, pc, o, jb, xs + slot * (uint32_t)kBlockBytes, lane);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl.blk_full[slot]);
      };
      plan.begin_item(it.nb);
      if (it.nb <= SlotPlan<F>::kS) {
        // the item fits: its units in order, slot of block b = b0 + b (ring)
        plan.begin_band(0);
        const uint32_t u0 = ucount, u1 = ucount + (uint32_t)(it.nb * kOctets);
        for (uint32_t u = u0 + ((uint32_t)gi + (uint32_t)kGenWarps - u0 % (uint32_t)kGenWarps) %
                                   (uint32_t)kGenWarps;
             u < u1; u += (uint32_t)kGenWarps) {
          const int b = (int)((u - u0) / (uint32_t)kOctets), o = (int)((u - u0) % (uint32_t)kOctets);
          const int slot = plan.slot_band(b);
          if (plan.used_band(b) &&
              !warp_wait(&ctl.blk_empty[slot], plan.parity_band(b) ^ 1u, &ctl, err, 64))
            goto gen_done;
          fill_octet(o, b, slot);
        }
        ucount = u1;
        continue;
      }
      plan.begin_item(it.nb);
      for (int r0 = 0; r0 < it.nb; r0 += plan.R()) {
        plan.begin_band(r0);
        for (int qb = 0; qb < it.nb - r0; ++qb, ucount += (uint32_t)kOctets) {
          int slot;
          uint32_t parity;
          bool used;
          if (qb < plan.Rb()) {
            slot = plan.slot_band(qb);
            parity = plan.parity_band(qb);
            used = plan.used_band(qb);
          } else {
            slot = plan.next_stream(parity, used);
          }
          const int jb = r0 + qb;     // column block of Phi
          bool waited = false;
          for (int o = (gi + kGenWarps - (int)(ucount % (uint32_t)kGenWarps)) % kGenWarps;
               o < kOctets; o += kGenWarps) {
            if (used && !waited) {
              if (!warp_wait(&ctl.blk_empty[slot], parity ^ 1u, &ctl, err, 64)) goto gen_done;
              waited = true;
            }
            fill_octet(o, jb, slot);
          }
        }
      }
    }
  gen_done:;
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kEpiWarps) {
    // --------------------------------------------------------- epilogue
    // All eight warps read every tile: warp w takes TMEM lanes 32(w%4) .. +31
    // (its rows of the tile) and the accumulator columns 64h .. 64h+63,
    // h = (w - 4) / 4, in two rounds of 32 Re and 32 Im columns (few, large
    // loads), and releases the buffer as soon as the second round's loads
    // have landed.  Tiles come in the MMA issuer's order (SlotPlan: each
    // band's triangle row by row, then its stream columns); only a band's
    // own triangle has diagonal tiles.
    const int qw = warp & 3;
    const int colh = 64 * ((warp - kEpiWarp0) >> 2);
    uint32_t gt = 0;
    SlotPlan<F> plan;
    for (int idx = blockIdx.x; idx < nitems; idx += gridDim.x) {
      ScreenItem it;
      if (!src.item(idx, t0, delta0, it)) continue;
      const int nb = it.nb;
      plan.begin_item(nb);
      float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      // one tile from accumulator buffer gt & 1; false if the wait gave up
      auto tile = [&](bool diag) -> bool {
        const uint32_t buf = gt & 1u, use = gt >> 1;
        ++gt;
        if (!warp_wait(&ctl.acc_full[buf], use & 1u, &ctl, err, 32)) return false;
        tc_fence_after();
        // the base is re-materialised per tile so the chunk addresses are
        // formed next to their loads instead of being held across the loop
        uint32_t base;
        asm volatile("mov.b32 %0, %1;" : "=r"(base) : "r"(tmem + ((uint32_t)(32 * qw) << 16) +
                                                          buf * 256u + (uint32_t)colh));
        if (!diag) {
          uint32_t ra[32], ia[32];
          tmem_ld32(base, ra);
          tmem_ld32(base + 128u, ia);
          tmem_wait_ld<32>(ra, ia);
          absmax<32>(ra, ia, m);
          tmem_ld32(base + 32u, ra);
          tmem_ld32(base + 160u, ia);
          tmem_wait_ld<32>(ra, ia);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl.acc_empty[buf]);
          absmax<32>(ra, ia, m);
          return true;
        }
        // diagonal tile: only column k > row j counts.  This warp's rows
        // are 32qw .. 32qw+31; a 16-column chunk n0 .. n0+15 lies entirely
        // at or below the diagonal (skip), entirely above it (no mask), or
        // straddles it (mask column n0 + e against row 32qw + lane).
        uint32_t ra[16], ia[16];
#pragma unroll 1
        for (int ch = 0; ch < 4; ++ch) {
          const int n0 = colh + 16 * ch;
          if (n0 + 16 <= 32 * qw) continue;
          tmem_ld16(base + 16u * ch, ra);
          tmem_ld16(base + 128u + 16u * ch, ia);
          tmem_wait_ld<16>(ra, ia);
          if (n0 >= 32 * qw + 32) {
            absmax<16>(ra, ia, m);
          } else {
            const int lim = 32 * qw + lane - n0;   // mask e <= lim
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float x = __uint_as_float(ra[e]), y = __uint_as_float(ia[e]);
              const float v = fmaf(x, x, y * y);
              m[e & 7] = (e > lim) ? fmaxf(m[e & 7], v) : m[e & 7];
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl.acc_empty[buf]);
        return true;
      };
      bool ok = true;
      if (nb <= SlotPlan<F>::kS) {
        int I = 0, J = 0;
        for (int tau = 0; tau < it.ntiles && ok; ++tau, J = (J + 1 < nb) ? J + 1 : ++I)
          ok = tile(I == J);
      }
      for (int r0 = 0; nb > SlotPlan<F>::kS && r0 < nb && ok; r0 += plan.R()) {
        const int Rb = min(plan.R(), nb - r0);
        for (int I = 0; I < Rb && ok; ++I)
          for (int J = I; J < Rb && ok; ++J) ok = tile(I == J);
        for (int J = Rb; J < nb - r0 && ok; ++J)
          for (int I = 0; I < Rb && ok; ++I) ok = tile(false);
      }
      if (!ok) break;
      float mx = fmaxf(fmax3(m[0], m[1], m[2]), fmax3(m[3], m[4], m[5]));
      mx = fmax3(mx, m[6], m[7]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) atomicMax(it.out, __float_as_uint(mx));
    }
  } else if (warp == kMmaWarp || warp == kMmaWarp2) {
    // ------------------------------------------------------ MMA issuers
    // Both walk the whole tile sequence, wait for every block, and commit
    // every slot release (blk_empty counts two commits); issuer iw issues the
    // tiles of accumulator buffer iw, i.e. the tiles gt with gt % 2 == iw.
    if (lane == 0) {
      const uint32_t iw = warp == kMmaWarp ? 0u : 1u;
      uint32_t gt = 0;
      SlotPlan<F> plan;
      const uint32_t hi = kDescHi;
      const uint32_t xs_lo = desc_lo(xs_addr);
      bool ok = true;
      auto issue_mmas = [&](uint32_t alo, uint32_t blo, uint32_t dre, uint32_t dim) {
        issue_tile_mmas<F>(alo, blo, dre, dim, hi);
      };
      auto tile = [&](int sA, int sB) -> bool {
        const uint32_t buf = gt & 1u, use = gt >> 1;
        ++gt;
        if (buf != iw) return true;
        if (use > 0 &&
            !mbar_wait(&ctl.acc_empty[buf], (use - 1u) & 1u, &ctl, err, kMmaBackoffNs))
          return false;
        tc_fence_after();
        const uint32_t alo = xs_lo + (uint32_t)sA * (uint32_t)(kBlockBytes >> 4);
        const uint32_t blo = xs_lo + (uint32_t)sB * (uint32_t)(kBlockBytes >> 4);
        const uint32_t dre = tmem + buf * 256u, dim = dre + 128u;
        issue_mmas(alo, blo, dre, dim);
        mma_commit(&ctl.acc_full[buf]);
        return true;
      };
      // Per band: its triangle row by row -- block I is last read in row I
      // (as A for J >= I, as B in rows I' <= I); the first row waits for each
      // block as it first needs it -- then, if blocks lie to its right, one
      // column of Rb tiles per stream block, after which the band's blocks
      // are released together.
      for (int idx = blockIdx.x; idx < nitems && ok; idx += gridDim.x) {
        ScreenItem it;
        if (!src.item(idx, t0, delta0, it)) continue;
        const int nb = it.nb;
        plan.begin_item(nb);
        if (nb <= SlotPlan<F>::kS) {
          // the item fits: row-major, slots of the ring advanced incrementally
          plan.begin_band(0);
          const int B = plan.B();
          uint32_t sI = (uint32_t)plan.slot_band(0);
          for (int I = 0; I < nb && ok; ++I, sI = (sI + 1 == (uint32_t)B) ? 0 : sI + 1) {
            const uint32_t alo = xs_lo + sI * (uint32_t)(kBlockBytes >> 4);
            uint32_t sJ = sI;
            for (int J = I; J < nb; ++J, ++gt, sJ = (sJ + 1 == (uint32_t)B) ? 0 : sJ + 1) {
              if (I == 0) {
                ok = mbar_wait(&ctl.blk_full[sJ], (plan.bsnap >> sJ) & 1u, &ctl, err,
                               kMmaBackoffNs);
                if (!ok) break;
              }
              const uint32_t buf = gt & 1u, use = gt >> 1;
              if (buf != iw) continue;
              if (use > 0) {
                ok = mbar_wait(&ctl.acc_empty[buf], (use - 1u) & 1u, &ctl, err, kMmaBackoffNs);
                if (!ok) break;
              }
              tc_fence_after();
              const uint32_t blo = xs_lo + sJ * (uint32_t)(kBlockBytes >> 4);
              const uint32_t dre = tmem + buf * 256u, dim = dre + 128u;
              issue_mmas(alo, blo, dre, dim);
              mma_commit(&ctl.acc_full[buf]);
            }
            if (ok) mma_commit(&ctl.blk_empty[sI]);   // row I done: block I's slot is free
          }
          continue;
        }
        for (int r0 = 0; r0 < nb && ok; r0 += plan.R()) {
          plan.begin_band(r0);
          const int Rb = plan.Rb();
          const bool stream = plan.streams();
          for (int I = 0; I < Rb && ok; ++I) {
            for (int J = I; J < Rb && ok; ++J) {
              if (I == 0) {
                ok = mbar_wait(&ctl.blk_full[plan.slot_band(J)], plan.parity_band(J), &ctl, err,
                               kMmaBackoffNs);
                if (!ok) break;
              }
              ok = tile(plan.slot_band(I), plan.slot_band(J));
            }
            if (ok && !stream) mma_commit(&ctl.blk_empty[plan.slot_band(I)]);   // row I done
          }
          if (!stream || !ok) continue;
          for (int qb = Rb; qb < nb - r0 && ok; ++qb) {
            uint32_t parity;
            bool used;
            const int sJ = plan.next_stream(parity, used);
            ok = mbar_wait(&ctl.blk_full[sJ], parity, &ctl, err, kMmaBackoffNs);
            for (int I = 0; I < Rb && ok; ++I) ok = tile(plan.slot_band(I), sJ);
            if (ok) mma_commit(&ctl.blk_empty[sJ]);
          }
          if (ok)
            for (int I = 0; I < Rb; ++I) mma_commit(&ctl.blk_empty[plan.slot_band(I)]);
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

// ------------------------------------------------------ survivor pair pass
// The precision form's preselection for the top-k re-score and for the
// certification: for each survivor s (candidate topk[s]) every tile of its
// upper-triangle Gram is formed again with the screen's operands and MMAs,
// one (survivor, tile) item per CTA at a time, and every pair whose screened
// |G_jk| is at least  mu_s - 2 err  is appended to the survivor's list, mu_s
// the survivor's screen score and err a bound on | |G|_screen - |G| | for any
// pair (|G| its binary32 or binary64 value).  The binary32 maximum pair of
// survivor s, and its binary64 one, lie within err of mu_s in the screen, so
// both are on the list; a list that would pass `cap` entries (or a bound that
// admits every pair) is marked by a count above cap, and *overflow_any is set.
struct PairPassArgs {
  ScreenArgs a;                 // frame, seed and round keys, sizes; a.st gates and
                                // gives the iteration's counter and radius
  const uint32_t* topk;         // survivor s -> candidate index
  const unsigned int* mu2;      // the K screen scores (float bits)
  int k;
  float err;
  uint2* pairs;                 // k x cap entries (j, k), j < k
  uint32_t* count;              // k counters (zero before the launch)
  uint32_t cap;
  uint32_t* overflow_any;
  // nullable: the survivors' column blocks drawn once by k_survivor_blocks
  // (survivor s, block b at (s nb + b) block sizes); else every item draws
  // its two blocks
  const unsigned char* blocks;
};

// The survivors' column blocks in the screen's operand layout, drawn once
// into global memory: one warp per (survivor, block, octet) unit, the
// screen's draw (gen_octet), so the pair pass only copies its two blocks.
template <int F>
__global__ void __launch_bounds__(256) k_survivor_blocks(const PairPassArgs p,
                                                         unsigned char* blocks) {
  constexpr int kBlockBytes = FmtTraits<F>::kBlockBytes;
  OneInstance src;
  src.a = p.a;
  uint32_t t0;
  float delta0;
  if (!src.launch(t0, delta0)) return;
  const int lane = threadIdx.x & 31;
  const int nb = p.a.nb, per = nb * kOctets;
  const int units = p.k * per;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); u < units; u += warps) {
    const int sv = u / per, rem = u - sv * per;
    const int b = rem / kOctets, o = rem - b * kOctets;
    ScreenItem it;
    it.N = p.a.N; it.d = p.a.d; it.nb = nb; it.ntiles = p.a.ntiles;
    it.phi = p.a.phi; it.seed = p.a.seed;
    it.cand = p.topk[sv]; it.t = t0; it.delta = delta0; it.out = nullptr;
    const PhiloxCand pc = src.cand(it);
    gen_octet<F>(src, it, pc, o, b, blocks + ((size_t)sv * nb + b) * kBlockBytes, lane);
  }
}

// 16 warps: all draw (one or two octets each per block pair), warp 0's lane 0
// issues the MMAs, and warp w reads tensor-memory lanes 32 (w % 4) .. +31 and
// accumulator columns 32 (w / 4) .. +31 of the tile.
constexpr int kPairWarps = 16;
template <int F>
__global__ void __launch_bounds__(32 * kPairWarps) k_screen_pairs(const PairPassArgs p) {
  constexpr int kBlockBytes = FmtTraits<F>::kBlockBytes;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ SmemCtl ctl;
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* xs = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t xs_addr = smem_u32(xs);
  OneInstance src;
  src.a = p.a;
  uint32_t t0;
  float delta0;
  if (!src.launch(t0, delta0)) return;   // iteration inactive or not screened
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* err = p.a.err;
  if (threadIdx.x == 0) {
    mbar_init(&ctl.acc_full[0], 1);
    mbar_init(&ctl.blk_full[0], 1);   // the two blocks' copies of an item
    ctl.abort_flag = 0;
    ctl.wait_limit_ns = kWaitLimitNs;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(&ctl.tmem_base)),
        "r"(256u)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl.tmem_base;
  const int ntiles = p.a.ntiles;
  const int nitems = p.k * ntiles;
  uint32_t phase = 0;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int sv = w / ntiles, tau = w - sv * ntiles;
    int I, J;
    tile_coords(tau, I, J);
    const uint32_t cand = p.topk[sv];
    const float lo = sqrtf(__uint_as_float(p.mu2[cand])) - 2.0f * p.err;
    if (!(lo > 0.0f)) {
      // the bound admits every pair: no list (the full passes decide)
      if (threadIdx.x == 0) {
        atomicMax(&p.count[sv], p.cap + 1u);
        atomicOr(p.overflow_any, 1u);
      }
      continue;
    }
    const float thr = __fmul_rd(lo, lo);
    ScreenItem it;
    it.N = p.a.N; it.d = p.a.d; it.nb = p.a.nb; it.ntiles = ntiles;
    it.phi = p.a.phi; it.seed = p.a.seed;
    it.cand = cand; it.t = t0; it.delta = delta0; it.out = nullptr;
    const int nblk = I == J ? 1 : 2;
    if (p.blocks) {
      // copy the item's blocks, drawn before
      if (threadIdx.x == 0) {
        const unsigned char* base = p.blocks + (size_t)sv * it.nb * kBlockBytes;
        mbar_expect_tx(&ctl.blk_full[0], (uint32_t)(nblk * kBlockBytes));
        bulk_g2s(xs, base + (size_t)I * kBlockBytes, (uint32_t)kBlockBytes, &ctl.blk_full[0]);
        if (nblk == 2)
          bulk_g2s(xs + kBlockBytes, base + (size_t)J * kBlockBytes, (uint32_t)kBlockBytes,
                   &ctl.blk_full[0]);
      }
      const bool got = warp_wait(&ctl.blk_full[0], phase, &ctl, err, 32);
      __syncthreads();
      if (!got || ctl.abort_flag) break;
    } else {
      const PhiloxCand pc = src.cand(it);
      for (int u = warp; u < nblk * kOctets; u += kPairWarps)
        gen_octet<F>(src, it, pc, u % kOctets, u < kOctets ? I : J,
                     xs + (u < kOctets ? 0u : (uint32_t)kBlockBytes), lane);
      fence_proxy_async_smem();
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t alo = desc_lo(xs_addr);
      const uint32_t blo = desc_lo(xs_addr + (nblk == 2 ? (uint32_t)kBlockBytes : 0u));
      issue_tile_mmas<F>(alo, blo, tmem, tmem + 128u, kDescHi);
      mma_commit(&ctl.acc_full[0]);
    }
    {
      const int qw = warp & 3, c0 = 32 * (warp >> 2);
      if (warp_wait(&ctl.acc_full[0], phase, &ctl, err, 32)) {
        tc_fence_after();
        const int row = 32 * qw + lane;
        const int j = I * kBlockCols + row;
        const uint32_t base = tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)c0;
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
          uint32_t ra[16], ia[16];
          tmem_ld16(base + 16u * ch, ra);
          tmem_ld16(base + 128u + 16u * ch, ia);
          tmem_wait_ld<16>(ra, ia);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float x = __uint_as_float(ra[e]), y = __uint_as_float(ia[e]);
            const float v = fmaf(y, y, x * x);
            const int col = c0 + 16 * ch + e;
            const int kk = J * kBlockCols + col;
            if (v >= thr && j < it.N && kk < it.N && (I != J || col > row)) {
              const uint32_t pos = atomicAdd(&p.count[sv], 1u);
              if (pos < p.cap)
                p.pairs[(size_t)sv * p.cap + pos] = make_uint2((uint32_t)j, (uint32_t)kk);
              else
                atomicOr(p.overflow_any, 1u);
            }
          }
        }
      }
    }
    phase ^= 1u;
    // the tile's tensor memory and shared-memory blocks are free again
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ctl.abort_flag) break;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                 : "memory");
}

// two blocks of the largest format and the 1 KiB alignment, at least 80 KiB so
// that at most two CTAs share an SM (2 x 256 tensor-memory columns)
constexpr size_t kPairPassSmem = 80 * 1024;
static_assert(kPairPassSmem >= 2 * 32768 + 1024, "pair pass blocks");

template <int F>
cudaError_t launch_pairs_fmt(const PairPassArgs& p, int grid, cudaStream_t s) {
  int fit = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &fit, k_screen_pairs<F>, 32 * kPairWarps, kPairPassSmem);
  if (e != cudaSuccess) return e;
  if (fit < 1) return cudaErrorLaunchOutOfResources;
  k_screen_pairs<F><<<grid, 32 * kPairWarps, kPairPassSmem, s>>>(p);
  return cudaGetLastError();
}

// the operand area is the same for every format: all slots of the ring
constexpr size_t kScreenSmem = (size_t)kOperandBytes + 1024;

template <class K> cudaError_t allow_screen_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              std::min((int)kScreenSmem, optin - (int)fa.sharedSizeBytes));
}

// refuse (without launching) a configuration the SM cannot hold
template <class K> cudaError_t screen_fits(K kernel) {
  int fit = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, kThreads, kScreenSmem);
  if (e != cudaSuccess) return e;
  return fit < 1 ? cudaErrorLaunchOutOfResources : cudaSuccess;
}

template <int F, class Src>
cudaError_t launch_fmt(const Src& src, int grid, cudaStream_t s) {
  cudaError_t e = screen_fits(k_screen<F, Src>);
  if (e != cudaSuccess) return e;
  // the operand area is always reserved for the whole ring, so every
  // descriptor address lies inside the CTA's shared memory
  k_screen<F, Src><<<grid, kThreads, kScreenSmem, s>>>(src);
  return cudaGetLastError();
}

template <class Src>
cudaError_t launch_any(int fmt, const Src& src, int grid, cudaStream_t s) {
  switch (fmt) {
    case kScreenBF16: return launch_fmt<kScreenBF16>(src, grid, s);
    case kScreenFP16: return launch_fmt<kScreenFP16>(src, grid, s);
    case kScreenTF32: return launch_fmt<kScreenTF32>(src, grid, s);
    case kScreenBF16W: return launch_fmt<kScreenBF16W>(src, grid, s);
    case kScreenFP16W: return launch_fmt<kScreenFP16W>(src, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Any N up to kScreenMaxN: beyond the ring (12 blocks of 128 columns, 6 for
// two-atom formats) the candidate is swept in bands (SlotPlan).
constexpr int kScreenMaxN = 65536;
// Bound on | |G|_screen - |G| | for one pair of unit columns, |G| its binary32
// or binary64 value: the operands' rounding (unit roundoff u: 2^-8 bf16,
// 2^-11 fp16 and tf32) moves a Gram entry by at most (2u + u^2) |phi_j| |phi_k|;
// 2^-12 covers, many times over, the rest (the screen's fast-math draw against
// the binary32 one, binary32 normalisation and fp32 accumulation, each a few
// 2^-24 per entry).
size_t screen_block_bytes(int fmt) {
  return (fmt == kScreenTF32 || fmt == kScreenBF16W || fmt == kScreenFP16W) ? 32768 : 16384;
}

float screen_pair_err(int fmt) {
  const double u = (fmt == kScreenBF16 || fmt == kScreenBF16W) ? 0.00390625 : 0.00048828125;
  return (float)(2.0 * u + u * u + 0.000244140625);
}

bool screen_supported(int N, int d, int fmt) {
  if (fmt < kScreenBF16 || fmt > kScreenFP16W) return false;
  const bool wide16 = fmt == kScreenBF16W || fmt == kScreenFP16W;
  return N >= 2 && N <= kScreenMaxN && d >= 1 && d <= (wide16 ? 64 : 32);
}

cudaError_t init_screen_attributes(int optin) {
  cudaError_t e;
  if ((e = allow_screen_smem(k_screen<kScreenBF16, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenFP16, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenTF32, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenBF16W, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenFP16W, OneInstance>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenBF16W, ManyInstances>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenFP16W, ManyInstances>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenBF16, ManyInstances>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenFP16, ManyInstances>, optin)) != cudaSuccess) return e;
  if ((e = allow_screen_smem(k_screen<kScreenTF32, ManyInstances>, optin)) != cudaSuccess) return e;
  const int pp = (int)kPairPassSmem;
  if ((e = cudaFuncSetAttribute(k_screen_pairs<kScreenBF16>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, pp)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_screen_pairs<kScreenFP16>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, pp)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_screen_pairs<kScreenTF32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, pp)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_screen_pairs<kScreenBF16W>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, pp)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_screen_pairs<kScreenFP16W>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, pp);
}

cudaError_t launch_screen(int fmt, int N, int d, uint64_t seed, const float2* phi32, int K,
                          uint32_t c0, uint32_t t, double delta, const DevState* st,
                          unsigned int* mu2_out, uint32_t* err_flag, int num_sms,
                          cudaStream_t s) {
  if (!screen_supported(N, d, fmt) || K < 1) return cudaErrorInvalidValue;
  OneInstance src;
  ScreenArgs& a = src.a;
  a.N = N; a.d = d;
  a.nb = (N + kBlockCols - 1) / kBlockCols;
  a.ntiles = a.nb * (a.nb + 1) / 2;
  a.K = K; a.seed = seed; a.phi = phi32; a.c0 = c0; a.t = t; a.delta = (float)delta;
  a.keys = philox_round_keys(seed);
  a.st = st; a.out = mu2_out; a.err = err_flag;
  a.wait_limit_ns = kWaitLimitNs;
  a.withhold_blocks = 0;
  return launch_any(fmt, src, std::min(K, num_sms), s);
}

cudaError_t launch_screen_pairs(int fmt, int N, int d, uint64_t seed, const float2* phi32,
                                const DevState* st, const uint32_t* topk,
                                const unsigned int* mu2, int k, float err, uint2* pairs,
                                uint32_t* count, uint32_t cap, uint32_t* overflow_any,
                                uint32_t* err_flag, int num_sms, cudaStream_t s,
                                unsigned char* blocks) {
  if (!screen_supported(N, d, fmt) || k < 1 || cap < 1) return cudaErrorInvalidValue;
  PairPassArgs p;
  ScreenArgs& a = p.a;
  a.N = N; a.d = d;
  a.nb = (N + kBlockCols - 1) / kBlockCols;
  a.ntiles = a.nb * (a.nb + 1) / 2;
  a.K = k; a.seed = seed; a.phi = phi32; a.c0 = 0; a.t = 0; a.delta = 0.f;
  a.keys = philox_round_keys(seed);
  a.st = st; a.out = nullptr; a.err = err_flag;
  a.wait_limit_ns = kWaitLimitNs;
  a.withhold_blocks = 0;
  p.topk = topk; p.mu2 = mu2; p.k = k; p.err = err;
  p.pairs = pairs; p.count = count; p.cap = cap; p.overflow_any = overflow_any;
  p.blocks = blocks;
  if (blocks) {
    const int warps = k * a.nb * kOctets;
    const int bgrid = std::max(1, std::min((warps + 7) / 8, 8 * num_sms));
    switch (fmt) {
      case kScreenBF16: k_survivor_blocks<kScreenBF16><<<bgrid, 256, 0, s>>>(p, blocks); break;
      case kScreenFP16: k_survivor_blocks<kScreenFP16><<<bgrid, 256, 0, s>>>(p, blocks); break;
      case kScreenTF32: k_survivor_blocks<kScreenTF32><<<bgrid, 256, 0, s>>>(p, blocks); break;
      case kScreenBF16W: k_survivor_blocks<kScreenBF16W><<<bgrid, 256, 0, s>>>(p, blocks); break;
      default: k_survivor_blocks<kScreenFP16W><<<bgrid, 256, 0, s>>>(p, blocks); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int grid = (int)std::min<long long>((long long)k * a.ntiles, 2LL * num_sms);
  switch (fmt) {
    case kScreenBF16: return launch_pairs_fmt<kScreenBF16>(p, grid, s);
    case kScreenFP16: return launch_pairs_fmt<kScreenFP16>(p, grid, s);
    case kScreenTF32: return launch_pairs_fmt<kScreenTF32>(p, grid, s);
    case kScreenBF16W: return launch_pairs_fmt<kScreenBF16W>(p, grid, s);
    case kScreenFP16W: return launch_pairs_fmt<kScreenFP16W>(p, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_screen_wait_test(int fmt, int N, int d, const float2* phi32, int K,
                                    unsigned int* mu2_out, uint32_t* err_flag,
                                    unsigned long long wait_limit_ns, int num_sms,
                                    cudaStream_t s) {
  if (!screen_supported(N, d, fmt) || K < 1 || wait_limit_ns == 0 ||
      wait_limit_ns > kWaitLimitNs)
    return cudaErrorInvalidValue;
  OneInstance src;
  ScreenArgs& a = src.a;
  a.N = N; a.d = d;
  a.nb = (N + kBlockCols - 1) / kBlockCols;
  a.ntiles = a.nb * (a.nb + 1) / 2;
  a.K = K; a.seed = 0; a.phi = phi32; a.c0 = 0; a.t = 1; a.delta = 0.f;
  a.keys = philox_round_keys(0);
  a.st = nullptr; a.out = mu2_out; a.err = err_flag;
  a.wait_limit_ns = wait_limit_ns;
  a.withhold_blocks = 1;
  return launch_any(fmt, src, std::min(K, num_sms), s);
}

cudaError_t launch_screen_batched(int fmt, const ScreenSlot* slots, const uint2* items,
                                  int n_items, uint32_t* err_flag, int num_sms, cudaStream_t s) {
  if (n_items < 1) return cudaSuccess;
  ManyInstances src;
  src.slots = slots;
  src.items = items;
  src.n_items = n_items;
  src.error = err_flag;
  return launch_any(fmt, src, std::min(n_items, num_sms), s);
}

}  // namespace trstmi
