// Device-side building blocks shared by the TensorACO kernels (sm_103a).
//
// Every floating-point operation whose result must be reproducible bit for
// bit uses an explicitly rounded intrinsic (__fmul_rn, __dadd_rn, ...), which
// the compiler never fuses into an FMA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tensoraco.h"

#define ACO_FULL_MASK 0xFFFFFFFFu

namespace aco {

// kernel-side check codes written to an instance's error word
constexpr int kErrConstruct = 1;     // an ant found no unvisited city
constexpr int kErrDepositRange = 2;  // deposit weights negative, NaN or spanning > 2^19
constexpr int kErrTimeout = 3;       // a bounded device-side wait ran out (reported as ACO_ERR_TIMEOUT)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// key += (W0, W1) between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a0 = c.x, a2 = c.z;
    const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of one Philox key, for callers that draw many blocks
// under it (an ant's whole walk): the key additions leave the per-draw chain.
struct PhiloxKeys {
  uint2 k[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint2 k) {
  PhiloxKeys ks;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    ks.k[r] = k;
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return ks;
}

// Round r (0..9) of Philox4x32-10 on counter block c, for callers that
// interleave the rounds with other work.
__device__ __forceinline__ void philox_round(uint4& c, const PhiloxKeys& ks, int r) {
  const uint32_t a0 = c.x, a2 = c.z;
  const uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
  const uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
  c = make_uint4(hi1 ^ c.y ^ ks.k[r].x, lo1, hi0 ^ c.w ^ ks.k[r].y, lo0);
}

__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKeys& ks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) philox_round(c, ks, r);
  return c;
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// r in (0,1): ((x >> 8) | 1) * 2^-24, exact.  Built without an int-to-float
// conversion: with a = x >> 9, the float 1 + a 2^-23 (a as its mantissa)
// minus (1 - 2^-24) is a 2^-23 + 2^-24 = (2a + 1) 2^-24, representable, so
// the single addition is exact.
__device__ __forceinline__ float uniform01(uint32_t x) {
  return __fadd_rn(__uint_as_float(0x3F800000u | (x >> 9)), 0x1p-24f - 1.0f);
}

// T_start of ant k: Lemire multiply-shift of word 0 of counter (0, 0, k, it).
__device__ __forceinline__ int start_city(uint2 key, uint32_t it, uint32_t k, int n) {
  uint4 w = philox(make_uint4(0u, 0u, k, it), key);
  return (int)(((uint64_t)w.x * (uint64_t)(uint32_t)n) >> 32);
}

// Integer power by left-to-right multiplication (a >= 0), each product rounded.
__device__ __forceinline__ float powi_f32(float x, int a) {
  if (a == 0) return 1.0f;
  float r = x;
  for (int i = 1; i < a; ++i) r = __fmul_rn(r, x);
  return r;
}
__device__ __forceinline__ double powi_f64(double x, int a) {
  if (a == 0) return 1.0;
  double r = x;
  for (int i = 1; i < a; ++i) r = __dmul_rn(r, x);
  return r;
}

// ---------------------------------------------------------------------------
// Own fp32 log2 / exp2 / pow for AdaIR's M_p^(1/gamma), from their series:
//   log2 x = k + (2/ln2) atanh(s), s = (mu-1)/(mu+1), mu in (sqrt(1/2), sqrt(2)],
//            atanh(s) = s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9)
//   2^y    = 2^i sum_{q=0..7} (f ln2)^q / q!,  i = rint(y), f = y - i
// Coefficients: fp32 roundings of 1/(2q+1), 2/ln 2, sqrt 2, (ln 2)^q / q!.
// ---------------------------------------------------------------------------
namespace own {
constexpr float kC3 = 0x1.555556p-2f;
constexpr float kC5 = 0x1.99999ap-3f;
constexpr float kC7 = 0x1.24924ap-3f;
constexpr float kC9 = 0x1.c71c72p-4f;
constexpr float kTwoOverLn2 = 0x1.715476p+1f;
constexpr float kSqrt2 = 0x1.6a09e6p+0f;
constexpr float kE1 = 0x1.62e430p-1f;
constexpr float kE2 = 0x1.ebfbe0p-3f;
constexpr float kE3 = 0x1.c6b08ep-5f;
constexpr float kE4 = 0x1.3b2ab6p-7f;
constexpr float kE5 = 0x1.5d87fep-10f;
constexpr float kE6 = 0x1.430912p-13f;
constexpr float kE7 = 0x1.ffcbfcp-17f;
}  // namespace own

__device__ __forceinline__ float log2_own(float x) {
  uint32_t b = __float_as_uint(x);
  int k = 0;
  if (((b >> 23) & 0xFF) == 0) {
    x = __fmul_rn(x, 0x1p23f);
    b = __float_as_uint(x);
    k = -23;
  }
  k += (int)((b >> 23) & 0xFF) - 127;
  float mu = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
  if (mu > own::kSqrt2) {
    mu = __fmul_rn(mu, 0.5f);
    k += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(mu, 1.0f), __fadd_rn(mu, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float q = own::kC9;
  q = __fadd_rn(__fmul_rn(q, s2), own::kC7);
  q = __fadd_rn(__fmul_rn(q, s2), own::kC5);
  q = __fadd_rn(__fmul_rn(q, s2), own::kC3);
  q = __fadd_rn(__fmul_rn(q, s2), 1.0f);
  const float l = __fmul_rn(__fmul_rn(s, q), own::kTwoOverLn2);
  return __fadd_rn((float)k, l);
}

// x * 2^i with at most one rounding (the last multiply).
__device__ __forceinline__ float scale_pow2(float x, int i) {
  if (i > 127) {
    x = __fmul_rn(x, 0x1p64f);
    i -= 64;
    if (i > 127) i = 128;
  }
  if (i < -126) {
    x = __fmul_rn(x, 0x1p-64f);
    i += 64;
    if (i < -126) {
      x = __fmul_rn(x, 0x1p-64f);
      i += 64;
    }
  }
  if (i == 128) return __fmul_rn(__fmul_rn(x, 0x1p127f), 2.0f);
  return __fmul_rn(x, __uint_as_float((uint32_t)(i + 127) << 23));
}

__device__ __forceinline__ float exp2_own(float y) {
  if (y != y) return y;
  if (y >= 129.0f) return __int_as_float(0x7F800000);
  if (y <= -151.0f) return 0.0f;
  const float fi = rintf(y);
  const float f = __fsub_rn(y, fi);
  float p = own::kE7;
  p = __fadd_rn(__fmul_rn(p, f), own::kE6);
  p = __fadd_rn(__fmul_rn(p, f), own::kE5);
  p = __fadd_rn(__fmul_rn(p, f), own::kE4);
  p = __fadd_rn(__fmul_rn(p, f), own::kE3);
  p = __fadd_rn(__fmul_rn(p, f), own::kE2);
  p = __fadd_rn(__fmul_rn(p, f), own::kE1);
  p = __fadd_rn(__fmul_rn(p, f), 1.0f);
  return scale_pow2(p, (int)fi);
}

__device__ __forceinline__ float pow_own(float x, float e) {
  if (x == 0.0f) return 0.0f;
  if (!(x < __int_as_float(0x7F800000))) return x;
  if (e == 1.0f) return x;
  return exp2_own(__fmul_rn(e, log2_own(x)));
}

}  // namespace aco
