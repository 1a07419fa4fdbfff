// Counter-based Gaussian draws for the candidate perturbation (device side).
//
// Philox4x32-10 is implemented here from its published definition (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
// ten rounds of two 32x32->64 multiplies with Weyl-sequence key bumps.
//
// Counter layout of this library (TRSTMI candidate step, the Monte-Carlo
// sampling of arXiv 2207.06374, Sec. "Optimization procedure"):
//   key = (seed lo32, seed hi32)
//   ctr = (e, c, t, tag),  e = j*ceil(d/2) + i/2  (entries i, i+1 of column j)
//   tag 0 = perturbation of iteration t, candidate c; tag 1 = initial frame.
// Each call yields u0..u3; U = (u + 1/2) 2^-32; entry i even uses (u0,u1),
// i odd (u2,u3); Z = sqrt(-ln Ua) * exp(2 pi i Ub) is complex normal CN(0,1)
// (the Box-Muller pair divided by sqrt 2).
#pragma once
#include <cstdint>

namespace trstmi {

struct PhiloxOut { uint32_t x[4]; };

__device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                   uint32_t c3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  constexpr uint32_t kBumpA = 0x9E3779B9u, kBumpB = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit product per multiplier gives both halves
    const uint64_t pA = (uint64_t)kMulA * (uint64_t)c0;
    const uint64_t pB = (uint64_t)kMulB * (uint64_t)c2;
    const uint32_t n0 = (uint32_t)(pB >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(pA >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)pB;
    c3 = (uint32_t)pA;
    c0 = n0; c2 = n2;
    k0 += kBumpA; k1 += kBumpB;
  }
  PhiloxOut o;
  o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
  return o;
}

// The ten round keys of one seed, (k0 + r W0, k1 + r W1), r = 0..9.
struct PhiloxKeys { uint32_t k0[10], k1[10]; };

__host__ __device__ inline PhiloxKeys philox_round_keys(uint64_t seed) {
  PhiloxKeys k;
  uint32_t a = (uint32_t)(seed & 0xffffffffull), b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = a; k.k1[r] = b;
    a += 0x9E3779B9u; b += 0xBB67AE85u;
  }
  return k;
}

// Same generator with the round keys given (e.g. from kernel parameters,
// which the instructions can read directly).
__device__ __forceinline__ PhiloxOut philox4x32_10_keys(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, const PhiloxKeys& k) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pA = (uint64_t)kMulA * (uint64_t)c0;
    const uint64_t pB = (uint64_t)kMulB * (uint64_t)c2;
    const uint32_t n0 = (uint32_t)(pB >> 32) ^ c1 ^ k.k0[r];
    const uint32_t n2 = (uint32_t)(pA >> 32) ^ c3 ^ k.k1[r];
    c1 = (uint32_t)pB;
    c3 = (uint32_t)pA;
    c0 = n0; c2 = n2;
  }
  PhiloxOut o;
  o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
  return o;
}

// Candidate-constant part of the first two rounds.  Within one candidate the
// counter words (c, t, 0) are fixed and only e varies, so round 1's product
// of the t word and round 2's product of the resulting word do not depend on
// e: they are formed once per candidate and each draw starts from them.
struct PhiloxCand {
  uint32_t c1k;   // round 2: low half of round 1's t product, xor round key k0[1]
  uint32_t c2k;   // round 2: high half of (mulA x round 1's first word) xor k1[1]
  uint32_t c3;    // round 2: low half of that product
};

__host__ __device__ inline PhiloxCand philox_cand(uint32_t c, uint32_t t, uint32_t k0_0,
                                                  uint32_t k0_1, uint32_t k1_1) {
  const uint64_t pB = (uint64_t)0xCD9E8D57u * (uint64_t)t;
  const uint32_t w0 = (uint32_t)(pB >> 32) ^ c ^ k0_0;       // round 1, first word
  const uint64_t pA = (uint64_t)0xD2511F53u * (uint64_t)w0;  // round 2 product of it
  PhiloxCand pc;
  pc.c1k = (uint32_t)pB ^ k0_1;
  pc.c2k = (uint32_t)(pA >> 32) ^ k1_1;
  pc.c3 = (uint32_t)pA;
  return pc;
}

// Philox4x32-10 of the counter (e, c, t, 0) from its candidate constants;
// k1_0 is the round-1 key k1, K0(r) / K1(r) give the keys of rounds r = 2..9.
template <class KeyFn>
__device__ __forceinline__ PhiloxOut philox_from_cand(uint32_t e, const PhiloxCand& pc,
                                                      uint32_t k1_0, KeyFn keys) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  const uint64_t p1 = (uint64_t)kMulA * (uint64_t)e;
  const uint32_t w2 = (uint32_t)(p1 >> 32) ^ k1_0;           // round 1, third word
  const uint64_t p2 = (uint64_t)kMulB * (uint64_t)w2;
  uint32_t c0 = (uint32_t)(p2 >> 32) ^ pc.c1k;
  uint32_t c1 = (uint32_t)p2;
  uint32_t c2 = pc.c2k ^ (uint32_t)p1;
  uint32_t c3 = pc.c3;
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    uint32_t k0, k1;
    keys(r, k0, k1);
    const uint64_t pA = (uint64_t)kMulA * (uint64_t)c0;
    const uint64_t pB = (uint64_t)kMulB * (uint64_t)c2;
    const uint32_t n0 = (uint32_t)(pB >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(pA >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)pB;
    c3 = (uint32_t)pA;
    c0 = n0; c2 = n2;
  }
  PhiloxOut o;
  o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
  return o;
}

// --- uniform -> complex normal, three precisions -------------------------

// Double precision: U = (u + 0.5) * 2^-32 is exact in binary64.
__device__ __forceinline__ void cn_from_u32_f64(uint32_t ua, uint32_t ub, double& re, double& im) {
  const double Ua = __dmul_rn(__dadd_rn((double)ua, 0.5), 0x1.0p-32);
  const double Ub = __dmul_rn(__dadd_rn((double)ub, 0.5), 0x1.0p-32);
  const double r = sqrt(-log(Ua));
  double s, c;
  sincospi(__dmul_rn(2.0, Ub), &s, &c);
  re = __dmul_rn(r, c);
  im = __dmul_rn(r, s);
}

// Single precision with the accurate library functions (plain FP32 path and
// the FP32 re-score of the screen survivors).
__device__ __forceinline__ void cn_from_u32_f32(uint32_t ua, uint32_t ub, float& re, float& im) {
  const float Ua = __fmaf_rn(__uint2float_rn(ua), 0x1.0p-32f, 0x1.0p-33f);
  const float Ub = __fmaf_rn(__uint2float_rn(ub), 0x1.0p-32f, 0x1.0p-33f);
  const float r = sqrtf(-logf(Ua));
  float s, c;
  sincospif(__fmul_rn(2.0f, Ub), &s, &c);
  re = __fmul_rn(r, c);
  im = __fmul_rn(r, s);
}

// Single precision with the hardware approximations; used only by the
// reduced-precision (bf16) screen, whose own rounding (2^-9) dominates.
// The angle is shifted into [-pi, pi) where the approximate sine/cosine are
// accurate: cos(2 pi U) = -cos(2 pi U - pi), likewise for the sine.
__device__ __forceinline__ void cn_from_u32_fast(uint32_t ua, uint32_t ub, float& re, float& im) {
  const float Ua = __fmaf_rn(__uint2float_rn(ua), 0x1.0p-32f, 0x1.0p-33f);
  const float Ub = __uint2float_rn(ub) * 0x1.0p-32f;
  // -ln U = -log2(U) * ln 2
  const float r = __fsqrt_rn(fmaxf(__log2f(Ua) * -0.69314718055994531f, 0.0f));
  const float th = __fmaf_rn(Ub, 6.28318530717958648f, -3.14159265358979324f);
  float s, c;
  __sincosf(th, &s, &c);
  re = -r * c;
  im = -r * s;
}

// Screen form of one perturbed entry: returns phi + delta * Z for the pair of
// words (ua, ub), with Z as in cn_from_u32_fast but cheaper: Ua by one
// conversion, the angle fraction Ub from the top 23 bits of ub placed in a
// float mantissa (f in [1, 2), Ub = f - 1, resolution 2^-23), and
// approximate lg2 / sqrt / sin / cos.
__device__ __forceinline__ void perturb_fast(uint32_t ua, uint32_t ub, float delta, float vr,
                                             float vi, float& xr, float& xi) {
  const float Ua = __fmaf_rn(__uint2float_rn(ua), 0x1.0p-32f, 0x1.0p-33f);
  float l2, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(Ua));
  const float e = fmaxf(l2 * -0.69314718055994531f, 0.0f);  // -ln Ua
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e));
  const float f = __int_as_float(0x3f800000u | (ub >> 9));
  // 2 pi Ub - pi = 2 pi f - 3 pi, in [-pi, pi); cos/sin(2 pi Ub) = -cos/sin of it
  const float th = __fmaf_rn(f, 6.28318530717958648f, -9.42477796076937972f);
  float s, c;
  __sincosf(th, &s, &c);
  const float dr = delta * r;
  xr = __fmaf_rn(-dr, c, vr);
  xi = __fmaf_rn(-dr, s, vi);
}

// Both entries of one draw (u0..u3) perturbed at once with paired binary32
// arithmetic, same approximations as perturb_fast: x0 = v0 + delta Z(u0, u1),
// x1 = v1 + delta Z(u2, u3).
__device__ __forceinline__ void perturb2_fast(const uint32_t (&u)[4], float delta, float2 v0,
                                              float2 v1, float2& x0, float2& x1) {
  const float2 Ua = __ffma2_rn(make_float2(__uint2float_rn(u[0]), __uint2float_rn(u[2])),
                               make_float2(0x1.0p-32f, 0x1.0p-32f),
                               make_float2(0x1.0p-33f, 0x1.0p-33f));
  float2 l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2.x) : "f"(Ua.x));
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2.y) : "f"(Ua.y));
  // sqrt(-ln U) = sqrt(ln 2) sqrt(|log2 U|); the factor sqrt(ln 2) joins the
  // radius below, and the magnitude guards a tiny positive approximation of
  // log2 near U = 1
  float2 r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(fabsf(l2.x)));
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(fabsf(l2.y)));
  const float2 f = make_float2(__int_as_float(0x3f800000u | (u[1] >> 9)),
                               __int_as_float(0x3f800000u | (u[3] >> 9)));
  const float2 th = __ffma2_rn(f, make_float2(6.28318530717958648f, 6.28318530717958648f),
                               make_float2(-9.42477796076937972f, -9.42477796076937972f));
  float s0, c0, s1, c1;
  __sincosf(th.x, &s0, &c0);
  __sincosf(th.y, &s1, &c1);
  const float ds = -delta * 0.83255461115769776f;   // -delta sqrt(ln 2)
  const float2 dr = __fmul2_rn(r, make_float2(ds, ds));
  x0 = __ffma2_rn(make_float2(dr.x, dr.x), make_float2(c0, s0), v0);
  x1 = __ffma2_rn(make_float2(dr.y, dr.y), make_float2(c1, s1), v1);
}

__device__ __forceinline__ uint32_t seed_lo(uint64_t s) { return (uint32_t)(s & 0xffffffffull); }
__device__ __forceinline__ uint32_t seed_hi(uint64_t s) { return (uint32_t)(s >> 32); }

}  // namespace trstmi
