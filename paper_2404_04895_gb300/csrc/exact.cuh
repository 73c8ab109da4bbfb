// Exact deposit arithmetic (Sec. 2.3, Eq. 3): the weights c_k = Q / L_k of
// the paths that use an edge are summed exactly in integer fixed point, and
// the evaporated pheromone plus that sum is rounded once to fp32.
//
// Fixed point.  Every positive finite double is M * 2^e with an integer
// M < 2^53.  With E0 the smallest e over the iteration's weights, weight k is
// the integer M_k << (e_k - E0) in units of 2^E0, at most 72 bits when the
// weights span at most kDepSpan binades.  It is held as three 24-bit chunks;
// per table entry, chunk q of every contributing weight is added into its own
// 64-bit word w_q (a carry-save form: no carries are propagated while
// summing, and 2^21 weights of < 2^24 cannot overflow a word).  Integer sums
// do not depend on their order, so the result is the same for any grouping
// or interleaving of the additions -- atomics included.
//
// Rounding.  tau' + (w0 + w1 2^24 + w2 2^48) 2^E0 is formed exactly in a
// 128-bit window whose top is the larger operand's leading bit (bits more
// than 100 places below it only set a sticky flag), then rounded to the
// nearest fp32, ties to even, with fp32's subnormal and overflow rules.
//
// Everything here is integer code, usable on the host as well, so that it
// can be checked against an independent exact summation on the CPU.
#pragma once

#include <stdint.h>

#include <cstring>

#if defined(__CUDACC__)
#define ACO_HD __host__ __device__ __forceinline__
#else
#define ACO_HD inline
#endif

namespace aco {

constexpr int kDepSpan = 19;  // binades the weights of one iteration may span (53 + 19 = 72 bits)

// deposit scaling modes; kDepNarrow: fixed point with every weight's
// exponent E0 or E0 + 1, so that a weight (at most 54 bits) is two 27-bit
// chunks instead of three 24-bit ones (32 of them still sum below 2^32)
enum { kDepFixed = 0, kDepInf = 1, kDepBad = 2, kDepNarrow = 3 };

ACO_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

ACO_HD uint64_t bits_of(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  std::memcpy(&b, &v, 8);
  return b;
#endif
}

ACO_HD uint32_t bits_of(float v) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(v);
#else
  uint32_t b;
  std::memcpy(&b, &v, 4);
  return b;
#endif
}

ACO_HD float float_of(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float v;
  std::memcpy(&v, &b, 4);
  return v;
#endif
}

// v = M * 2^e for a positive finite double (M < 2^53; subnormals included)
ACO_HD void split_double(double v, uint64_t* M, int* e) {
  const uint64_t b = bits_of(v);
  const int eb = (int)((b >> 52) & 0x7FF);
  *M = (b & 0xFFFFFFFFFFFFFull) | (eb ? (1ull << 52) : 0ull);
  *e = (eb ? eb : 1) - 1075;
}

// exponent e of a positive finite double (as in split_double)
ACO_HD int exponent_of(double v) {
  const int eb = (int)((bits_of(v) >> 52) & 0x7FF);
  return (eb ? eb : 1) - 1075;
}

// The three 24-bit chunks of weight v in units of 2^E0 (v positive finite,
// exponent_of(v) - E0 in [0, kDepSpan]).
ACO_HD void weight_chunks(double v, int E0, uint32_t* c0, uint32_t* c1, uint32_t* c2) {
  uint64_t M;
  int e;
  split_double(v, &M, &e);
  const int s = e - E0;
  const uint64_t lo = M << s;
  const uint64_t hi = s ? (M >> (64 - s)) : 0ull;
  *c0 = (uint32_t)(lo & 0xFFFFFFull);
  *c1 = (uint32_t)((lo >> 24) & 0xFFFFFFull);
  *c2 = (uint32_t)((lo >> 48) | (hi << 16));
}

// The two 27-bit chunks of weight v in units of 2^E0 (v positive finite,
// exponent_of(v) - E0 in {0, 1}: at most 54 bits).  Chunk 1 counts units of
// 2^(E0 + 27), i.e. (c1 << 3) units of 2^(E0 + 24) in the three-chunk form.
ACO_HD void weight_chunks27(double v, int E0, uint32_t* c0, uint32_t* c1) {
  uint64_t M;
  int e;
  split_double(v, &M, &e);
  const uint64_t w = M << (e - E0);
  *c0 = (uint32_t)(w & 0x7FFFFFFull);
  *c1 = (uint32_t)(w >> 27);
}

// (hi, lo) += (bh, bl)
ACO_HD void add128(uint64_t* hi, uint64_t* lo, uint64_t bh, uint64_t bl) {
  const uint64_t l = *lo + bl;
  *hi += bh + (l < bl ? 1ull : 0ull);
  *lo = l;
}

// (hi, lo) * 2^s for s >= 0 (the caller guarantees no bit leaves the top),
// or / 2^-s for s < 0 with every dropped bit ORed into *sticky.
ACO_HD void shift128(uint64_t hi, uint64_t lo, int s, uint64_t* oh, uint64_t* ol, bool* sticky) {
  if (s >= 0) {
    if (s >= 64) {
      *oh = lo << (s - 64);
      *ol = 0ull;
    } else if (s > 0) {
      *oh = (hi << s) | (lo >> (64 - s));
      *ol = lo << s;
    } else {
      *oh = hi;
      *ol = lo;
    }
    return;
  }
  const int r = -s;
  if (r >= 128) {
    if (hi | lo) *sticky = true;
    *oh = 0ull;
    *ol = 0ull;
  } else if (r >= 64) {
    const int q = r - 64;
    if (lo || (q && (hi << (64 - q)))) *sticky = true;
    *ol = q ? (hi >> q) : hi;
    *oh = 0ull;
  } else {
    if (lo << (64 - r)) *sticky = true;
    *ol = (lo >> r) | (hi << (64 - r));
    *oh = hi >> r;
  }
}

// index of the highest set bit of a nonzero (hi, lo)
ACO_HD int top128(uint64_t hi, uint64_t lo) { return hi ? 127 - clz64(hi) : 63 - clz64(lo); }

// bit p (0..127) of (hi, lo)
ACO_HD uint64_t bit128(uint64_t hi, uint64_t lo, int p) { return p >= 64 ? (hi >> (p - 64)) & 1ull : (lo >> p) & 1ull; }

// any bit below position p (0..128) of (hi, lo)
ACO_HD bool any_below128(uint64_t hi, uint64_t lo, int p) {
  if (p <= 0) return false;
  if (p >= 128) return (hi | lo) != 0ull;
  if (p >= 64) return lo != 0ull || (p > 64 && (hi << (128 - p)) != 0ull);
  return (lo << (64 - p)) != 0ull;
}

// The number nearest to tp + (w0 + w1 2^24 + w2 2^48) 2^E0 (ties to even) in
// a binary format with MB significant bits and fp32's exponent range (MB =
// 24: fp32; MB = 8: bfloat16), returned as its fp32 bit pattern, for tp >= 0
// (+inf allowed) and an exact nonnegative fixed-point sum.
template <int MB>
ACO_HD uint32_t round_sum_bits(float tp, uint64_t w0, uint64_t w1, uint64_t w2, int E0) {
  constexpr int LSB_MIN = -126 - (MB - 1);  // exponent of the smallest subnormal
  uint64_t ah = 0ull, al = w0;
  add128(&ah, &al, w1 >> 40, w1 << 24);
  add128(&ah, &al, w2 >> 16, w2 << 48);
  const uint32_t tb = bits_of(tp);
  if ((ah | al) == 0ull && MB == 24) return tb;
  const int teb = (int)(tb >> 23);
  if (teb >= 255) return tb;  // +inf stays +inf
  const uint64_t mt = (uint64_t)(tb & 0x7FFFFFu) | (teb ? 0x800000ull : 0ull);
  if ((ah | al) == 0ull && mt == 0ull) return 0u;
  const int et = (teb ? teb : 1) - 150;
  // leading-bit exponent of the larger operand; window LSB 100 places below it
  int T = (ah | al) ? top128(ah, al) + E0 : -100000;
  if (mt) {
    const int tt = 63 - clz64(mt) + et;
    T = tt > T ? tt : T;
  }
  const int base = T - 100;
  bool sticky = false;
  uint64_t sh = 0ull, sl = 0ull;
  if (ah | al) shift128(ah, al, E0 - base, &sh, &sl, &sticky);
  if (mt) {
    uint64_t mh, ml;
    shift128(0ull, mt, et - base, &mh, &ml, &sticky);
    add128(&sh, &sl, mh, ml);
  }
  // keep the bits from position r up: MB significant bits, or down to 2^LSB_MIN
  const int top = top128(sh, sl);
  int r = top - (MB - 1);
  if (LSB_MIN - base > r) r = LSB_MIN - base;
  if (r > 128) return 0u;  // far below the smallest subnormal
  uint64_t mant_h, mant_l;
  bool dummy = false;
  shift128(sh, sl, -r, &mant_h, &mant_l, &dummy);
  uint64_t mant = mant_l;  // < 2^MB
  const uint64_t round_bit = r >= 1 ? bit128(sh, sl, r - 1) : 0ull;
  const bool below = sticky || any_below128(sh, sl, r - 1);
  if (round_bit && (below || (mant & 1ull))) mant += 1ull;
  int e_lsb = r + base;  // exponent of the kept LSB
  if (mant >> MB) {      // carried into one more bit
    mant >>= 1;
    e_lsb += 1;
  }
  if (mant == 0ull) return 0u;
  if (mant < (1ull << (MB - 1))) return (uint32_t)(mant << (LSB_MIN + 149));  // subnormal (e_lsb = LSB_MIN)
  const int E = e_lsb + (MB - 1) + 127;                                        // biased exponent
  if (E >= 255) return 0x7F800000u;
  return ((uint32_t)E << 23) | ((uint32_t)(mant & ((1ull << (MB - 1)) - 1ull)) << (24 - MB));
}

// The fp32 nearest to tp + (w0 + w1 2^24 + w2 2^48) 2^E0 (ties to even).
ACO_HD float round_sum_f32(float tp, uint64_t w0, uint64_t w1, uint64_t w2, int E0) {
  return float_of(round_sum_bits<24>(tp, w0, w1, w2, E0));
}

// The bfloat16 nearest to the same sum (ties to even), as its 16-bit pattern.
ACO_HD uint32_t round_sum_bf16(float tp, uint64_t w0, uint64_t w1, uint64_t w2, int E0) {
  return round_sum_bits<8>(tp, w0, w1, w2, E0) >> 16;
}

}  // namespace aco
