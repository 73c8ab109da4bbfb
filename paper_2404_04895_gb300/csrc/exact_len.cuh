// Exact tour length (Eq. 3): f(s) is the plain sum of the tour's n fp64 edge
// lengths; it is taken exactly and rounded once to fp64 (ties to even), so
// the result depends on no order of the edges and any split of a tour across
// lanes, warps or blocks gives the same bits.
//
// Fixed point.  An edge length computed from fp32 coordinates,
// d = sqrt(dx^2 + dy^2) in fp64, is either 0 or lies in [2^-149, 2^130): a
// nonzero fp32 difference is at least 2^-149 and at most 2^129 in magnitude.
// Such a d is M * 2^e with an integer M < 2^53 and e >= -201, i.e. the integer
// M << (e + 201) in units of 2^-201, below 2^331.  A tour of n <= 2^16 edges
// sums to less than 2^347: eleven 32-bit digits.  A partial sum keeps each
// digit in its own 64-bit word (a carry-save form: adding a < 2^32 chunk per
// edge, 2^32 edges could not overflow a word), so an edge costs three
// independent integer adds and no carry chain; digits are normalised only
// when partial sums are combined and rounded.
//
// Everything here is integer code, usable on the host as well, so that it
// can be checked against an independent exact summation on the CPU.
#pragma once

#include <stdint.h>

#include "exact.cuh"

namespace aco {

constexpr int kLenDigits = 11;     // 32-bit digits of a tour-length sum (352 bits)
constexpr int kLenUnitExp = -201;  // the accumulator counts units of 2^-201
constexpr int kLenMinBiased = 874;   // biased exponent of 2^-149: the smallest nonzero edge
constexpr int kLenMaxBiased = 1152;  // biased exponent of [2^129, 2^130): the largest edge

// True for the edge lengths the accumulator holds exactly: +0 or a positive
// double in [2^-149, 2^130) (bit pattern b).
ACO_HD bool len_in_range(uint64_t b) {
  const uint32_t eb = (uint32_t)(b >> 52);  // the sign bit makes eb >= 2048
  return b == 0ull || (eb >= (uint32_t)kLenMinBiased && eb <= (uint32_t)kLenMaxBiased);
}

// The digits of a nonzero in-range edge length with bit pattern b: d is
// (w0 + w1 2^32 + w2 2^64) units of 2^-201 times 2^(32 q); returns q (0..8,
// so q + 2 is a digit of the sum).
ACO_HD int len_digits(uint64_t b, uint32_t* w0, uint32_t* w1, uint32_t* w2) {
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int s = (int)(b >> 52) - kLenMinBiased;  // [0, 278]
  const int r = s & 31;
  const uint64_t lo = M << r;
  *w0 = (uint32_t)lo;
  *w1 = (uint32_t)(lo >> 32);
  *w2 = r ? (uint32_t)(M >> (64 - r)) : 0u;
  return s >> 5;
}

// acc += d for an in-range edge length with bit pattern b.
ACO_HD void len_acc_add(uint64_t acc[kLenDigits], uint64_t b) {
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int s = (int)(b >> 52) - kLenMinBiased;  // shift of M in units of 2^-201: [0, 278]
  const int q = s >> 5, r = s & 31;
  const uint64_t lo = M << r;
  uint32_t w0 = (uint32_t)lo, w1 = (uint32_t)(lo >> 32);
  uint32_t w2 = r ? (uint32_t)(M >> (64 - r)) : 0u;
  if (b == 0ull) w0 = w1 = w2 = 0u;  // a zero edge (coincident cities)
#pragma unroll
  for (int i = 0; i < kLenDigits; ++i) {
    const int t = i - q;
    acc[i] += t == 0 ? w0 : (t == 1 ? w1 : (t == 2 ? w2 : 0u));
  }
}

// Fast window.  One instance's edge lengths span few binades, so nearly every
// edge of a tour starts at digit kLenWin or kLenWin + 1 (d in [2^-21, 2^43)).
// Such an edge goes into a four-digit window (digits kLenWin .. kLenWin + 3)
// with two-way selects instead of the full accumulator's eleven; any other
// edge goes to the full accumulator, and len_win_merge adds the window back.
// Integer sums again: the total is the same bits.
constexpr int kLenWin = 4;

// win += d and true if the in-range edge length with bit pattern b is 0 or
// starts at digit kLenWin or kLenWin + 1; else win unchanged and false.
ACO_HD bool len_win_add(uint64_t win[4], uint64_t b) {
  if (b == 0ull) return true;
  const int s = (int)(b >> 52) - kLenMinBiased;
  const int t = (s >> 5) - kLenWin;
  if ((unsigned)t > 1u) return false;
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int r = s & 31;
  const uint64_t lo = M << r;
  const uint32_t w0 = (uint32_t)lo, w1 = (uint32_t)(lo >> 32);
  const uint32_t w2 = r ? (uint32_t)(M >> (64 - r)) : 0u;
  const bool z = t == 0;
  win[0] += z ? w0 : 0u;
  win[1] += z ? w1 : w0;
  win[2] += z ? w2 : w1;
  win[3] += z ? 0u : w2;
  return true;
}

// acc += the window (before len_acc_carry).
ACO_HD void len_win_merge(uint64_t acc[kLenDigits], const uint64_t win[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[kLenWin + i] += win[i];
}

// The window as five digits below 2^32 (the fifth takes the carry out of the
// fourth), digit kLenWin + i in out[i]; the same value.
ACO_HD void len_win_digits(const uint64_t win[4], uint64_t out[5]) {
  uint64_t carry = 0ull;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t v = win[i] + carry;  // win[i] < 2^48: no overflow
    out[i] = v & 0xFFFFFFFFull;
    carry = v >> 32;
  }
  out[4] = carry;
}

// Carry propagation: afterwards every digit but the last is < 2^32 and the
// value is unchanged (the last holds the rest: < 2^27 for any tour sum).
ACO_HD void len_acc_carry(uint64_t acc[kLenDigits]) {
#pragma unroll
  for (int i = 0; i + 1 < kLenDigits; ++i) {
    acc[i + 1] += acc[i] >> 32;
    acc[i] &= 0xFFFFFFFFull;
  }
}

// The double nearest to the accumulated sum (ties to even).  acc is any
// carry-save form of the sum (it is normalised in place).
ACO_HD double len_acc_round(uint64_t acc[kLenDigits]) {
  len_acc_carry(acc);
  // a 96-bit window of digits top, top-1, top-2 (top: the highest nonzero
  // digit; missing digits are 0) and a sticky flag for every digit below it,
  // gathered in one pass from the top (no digit is picked by a run-time index)
  int top = -1, taken = 0;
  uint64_t d2 = 0ull, d1 = 0ull, d0 = 0ull;
  bool sticky = false;
#pragma unroll
  for (int i = kLenDigits - 1; i >= 0; --i) {
    const uint64_t v = acc[i];
    if (top < 0) {
      if (v) {
        top = i;
        d2 = v;
      }
    } else if (taken == 0) {
      d1 = v;
      taken = 1;
    } else if (taken == 1) {
      d0 = v;
      taken = 2;
    } else if (v) {
      sticky = true;
    }
  }
  if (top < 0) return 0.0;
  const uint64_t hi = (d2 << 32) | d1;  // window bits 32..95; d0 holds bits 0..31
  const int tb = 95 - clz64(hi);         // the window's leading bit: 64..95
  const int k = tb - 52;                 // the kept 53 bits are window bits k..tb
  uint64_t mant;
  bool rbit, rest;
  if (k >= 32) {
    mant = hi >> (k - 32);
    const int rp = k - 33;  // the round bit's place in hi (k >= 33) or d0's bit 31
    if (rp >= 0) {
      rbit = (hi >> rp) & 1ull;
      rest = d0 != 0ull || (rp > 0 && (hi << (64 - rp)) != 0ull);
    } else {
      rbit = (d0 >> 31) & 1ull;
      rest = (d0 & 0x7FFFFFFFull) != 0ull;
    }
  } else {
    mant = (hi << (32 - k)) | (d0 >> k);
    rbit = (d0 >> (k - 1)) & 1ull;
    rest = (d0 & ((1ull << (k - 1)) - 1ull)) != 0ull;
  }
  if (rbit && (rest || sticky || (mant & 1ull))) mant += 1ull;
  int e_unit = k + 32 * (top - 2) + kLenUnitExp;  // exponent of mant's last bit
  if (mant >> 53) {
    mant >>= 1;
    e_unit += 1;
  }
  const uint64_t E = (uint64_t)(e_unit + 52 + 1023);  // a normal double: the sum is >= 2^-149
  const uint64_t bits = (E << 52) | (mant & 0xFFFFFFFFFFFFFull);
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)bits);
#else
  double v;
  std::memcpy(&v, &bits, 8);
  return v;
#endif
}

}  // namespace aco
