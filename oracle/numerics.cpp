// TensorACO CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// Random numbers, IEEE rounding to 16-bit formats, integer powers and the
// own-polynomial pow used by AdaIR.  Compiled with -O2 -ffp-contract=off so
// that every product and sum is rounded on its own, as written.
#include "oracle.h"

#include <cmath>
#include <cstring>

namespace {

uint32_t f2u(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
float u2f(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Philox4x32 constants (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5):
// round multipliers and the Weyl key increments (golden ratio, sqrt(3)-1).
const uint32_t PHILOX_M0 = 0xD2511F53u;
const uint32_t PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u;
const uint32_t PHILOX_W1 = 0xBB67AE85u;

// x >> s rounded to nearest, ties to even (s >= 1).
uint64_t shift_right_rne(uint64_t x, int s) {
  if (s >= 64) return 0;
  uint64_t q = x >> s;
  uint64_t rem = x - (q << s);
  uint64_t half = (uint64_t)1 << (s - 1);
  if (rem > half || (rem == half && (q & 1))) q += 1;
  return q;
}

}  // namespace

extern "C" {

// One Philox4x32-10 block: ten rounds of the S-box
//   (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
// with the key bumped by (W0, W1) between rounds.
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// The random deviate for candidate j at step t of ant k, iteration it
// (Sec. 2.4: one independent uniform per candidate city).
uint32_t orc_draw(uint64_t seed, uint32_t it, uint32_t k, uint32_t t, uint32_t j) {
  uint32_t ctr[4] = {j >> 2, t, k, it};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[j & 3];
}

// r in (0,1): the top 24 bits of x with the lowest forced to one, times 2^-24.
// Both steps are exact in fp32.
float orc_uniform(uint32_t x) {
  uint32_t k24 = (x >> 8) | 1u;
  return (float)k24 * 0x1p-24f;
}

// T_start (Sec. 2.2): a uniform city index in [0, n) from word 0 of the
// step-0 counter, by Lemire's multiply-shift.
int32_t orc_start_city(uint64_t seed, uint32_t it, uint32_t k, int32_t n) {
  uint32_t ctr[4] = {0u, 0u, k, it};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return (int32_t)(((uint64_t)out[0] * (uint64_t)(uint32_t)n) >> 32);
}

// fp32 -> bfloat16, round to nearest even (IEEE-754 semantics on the 8-bit
// exponent, 7-bit fraction format).
uint16_t orc_to_bf16(float x) {
  uint32_t b = f2u(x);
  uint32_t sign = b & 0x80000000u;
  uint32_t mag = b & 0x7FFFFFFFu;
  if (mag > 0x7F800000u) return (uint16_t)((b >> 16) | 0x0040u);  // quiet NaN
  // keep 16 high bits of the magnitude, round the dropped 16 bits
  uint64_t q = shift_right_rne(mag, 16);  // may carry into the exponent: correct
  return (uint16_t)((sign >> 16) | (uint32_t)q);
}

float orc_from_bf16(uint16_t h) { return u2f((uint32_t)h << 16); }

// fp32 -> IEEE binary16, round to nearest even, with subnormals and overflow to
// infinity, written from the format's definition.
uint16_t orc_to_fp16(float x) {
  uint32_t b = f2u(x);
  uint16_t sign = (uint16_t)((b >> 16) & 0x8000u);
  int ef = (int)((b >> 23) & 0xFF);
  uint32_t frac = b & 0x7FFFFFu;
  if (ef == 0xFF) return (uint16_t)(sign | 0x7C00u | (frac ? 0x200u : 0u));
  if (ef == 0) return sign;  // fp32 zero or subnormal (< 2^-126): rounds to zero
  int e = ef - 127;                          // value = m * 2^(e-23), m in [2^23, 2^24)
  uint64_t m = (uint64_t)(frac | 0x800000u);
  if (e >= -14) {
    // normal binary16: 11 significant bits
    uint64_t q = shift_right_rne(m, 13);     // in [2^10, 2^11]
    if (q == (1u << 11)) {
      q >>= 1;
      e += 1;
    }
    int he = e + 15;
    if (he >= 31) return (uint16_t)(sign | 0x7C00u);
    return (uint16_t)(sign | (uint16_t)(he << 10) | (uint16_t)(q & 0x3FFu));
  }
  // subnormal binary16: value in units of 2^-24 is m * 2^(e+1)
  int s = -(e + 1);                          // >= 14
  uint64_t q = shift_right_rne(m, s);        // may reach 0x400: smallest normal
  return (uint16_t)(sign | (uint16_t)q);
}

float orc_from_fp16(uint16_t h) {
  uint32_t sign = ((uint32_t)h & 0x8000u) << 16;
  int e = (h >> 10) & 0x1F;
  uint32_t f = h & 0x3FFu;
  if (e == 0x1F) return u2f(sign | 0x7F800000u | (f << 13));
  if (e == 0) {
    float v = (float)f * 0x1p-24f;  // exact
    return sign ? -v : v;
  }
  return u2f(sign | (uint32_t)(e - 15 + 127) << 23 | (f << 13));
}

void orc_to_bf16_array(const float* x, uint16_t* out, int64_t count) {
  for (int64_t i = 0; i < count; ++i) out[i] = orc_to_bf16(x[i]);
}
void orc_to_fp16_array(const float* x, uint16_t* out, int64_t count) {
  for (int64_t i = 0; i < count; ++i) out[i] = orc_to_fp16(x[i]);
}

// x^a for an integer a >= 0: 1 for a = 0, else x*x*...*x left to right,
// each product rounded (a-1 roundings).
float orc_powi_f32(float x, int a) {
  if (a == 0) return 1.0f;
  float r = x;
  for (int i = 1; i < a; ++i) r = r * x;
  return r;
}
double orc_powi_f64(double x, int a) {
  if (a == 0) return 1.0;
  double r = x;
  for (int i = 1; i < a; ++i) r = r * x;
  return r;
}

// ---- own log2 / exp2 (fp32), written from their series ----
//
// log2(x) = k + (2/ln 2) * atanh(s),  x = mu * 2^k, mu in (sqrt(1/2), sqrt(2)],
//           s = (mu - 1) / (mu + 1),  atanh(s) = s * (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9)
// 2^y     = 2^i * exp(f ln 2),        i = round-to-even(y), f = y - i in [-1/2, 1/2],
//           exp(z) = sum_{q=0..7} z^q / q!
// The fp32 coefficients are rounded once from fp64 values of 1/(2q+1), 2/ln 2,
// (ln 2)^q / q! and sqrt(2).

namespace {
struct OwnCoeffs {
  float c3, c5, c7, c9, two_over_ln2, sqrt2;
  float e[8];
  OwnCoeffs() {
    c3 = (float)(1.0 / 3.0);
    c5 = (float)(1.0 / 5.0);
    c7 = (float)(1.0 / 7.0);
    c9 = (float)(1.0 / 9.0);
    double ln2 = std::log(2.0);
    two_over_ln2 = (float)(2.0 / ln2);
    sqrt2 = (float)std::sqrt(2.0);
    double fact = 1.0;
    for (int q = 0; q < 8; ++q) {
      if (q > 0) fact = fact * (double)q;
      e[q] = (float)(orc_powi_f64(ln2, q) / fact);
    }
  }
};
const OwnCoeffs& coeffs() {
  static const OwnCoeffs c;
  return c;
}

// x * 2^i for |i| possibly beyond the fp32 exponent range: at most one rounding.
float scale_pow2(float x, int i) {
  if (i > 127) {
    x = x * 0x1p64f;
    i -= 64;
    if (i > 127) i = 127 + 1;  // overflows below
  }
  if (i < -126) {
    x = x * 0x1p-64f;
    i += 64;
    if (i < -126) {
      x = x * 0x1p-64f;
      i += 64;
    }
  }
  if (i == 128) return x * 0x1p127f * 2.0f;
  return x * u2f((uint32_t)(i + 127) << 23);
}
}  // namespace

float orc_log2_own(float x) {
  const OwnCoeffs& c = coeffs();
  uint32_t b = f2u(x);
  int k = 0;
  if (((b >> 23) & 0xFF) == 0) {  // subnormal: scale into the normal range
    x = x * 0x1p23f;
    b = f2u(x);
    k = -23;
  }
  k += (int)((b >> 23) & 0xFF) - 127;
  float mu = u2f((b & 0x7FFFFFu) | 0x3F800000u);  // [1, 2)
  if (mu > c.sqrt2) {
    mu = mu * 0.5f;
    k += 1;
  }
  float s = (mu - 1.0f) / (mu + 1.0f);
  float s2 = s * s;
  float q = c.c9;
  q = q * s2 + c.c7;
  q = q * s2 + c.c5;
  q = q * s2 + c.c3;
  q = q * s2 + 1.0f;
  float log2mu = (s * q) * c.two_over_ln2;
  return (float)k + log2mu;
}

float orc_exp2_own(float y) {
  const OwnCoeffs& c = coeffs();
  if (y != y) return y;
  if (y >= 129.0f) return INFINITY;
  if (y <= -151.0f) return 0.0f;
  float fi = std::nearbyint(y);  // default rounding mode: to nearest, ties to even
  float f = y - fi;              // exact, |f| <= 1/2
  float p = c.e[7];
  for (int q = 6; q >= 0; --q) p = p * f + c.e[q];
  return scale_pow2(p, (int)fi);
}

// x^e for x >= 0 (Sec. 2.4: AdaIR's exponent applied to M_p).
float orc_pow_own(float x, float e) {
  if (x == 0.0f) return 0.0f;
  if (!(x < INFINITY)) return x;
  if (e == 1.0f) return x;
  return orc_exp2_own(e * orc_log2_own(x));
}

void orc_pow_own_array(const float* x, float e, float* out, int64_t count) {
  for (int64_t i = 0; i < count; ++i) out[i] = orc_pow_own(x[i], e);
}

// Cosine-annealing schedule for AdaIR's gamma (Sec. 2.4), evaluated in fp64
// and rounded to fp32:  gamma_t = g_min + (g_max - g_min)/2 * (1 + cos(pi t / T))
// for t < T, and g_min afterwards.
float orc_gamma(int it, int T, float gamma_max, float gamma_min) {
  if (T <= 0 || it >= T) return gamma_min;
  double gmax = (double)gamma_max, gmin = (double)gamma_min;
  double ang = 3.14159265358979323846 * (double)it / (double)T;
  double g = gmin + 0.5 * (gmax - gmin) * (1.0 + std::cos(ang));
  return (float)g;
}

float orc_inv_gamma(float gamma) { return (float)(1.0 / (double)gamma); }

double orc_adair_deviate(double r, double gamma) { return std::pow(r, gamma); }

}  // extern "C"
