// Host build of the library's exact arithmetic for the CPU tests:
//   - the deposit (csrc/exact.cuh, the integer code the deposit kernel runs):
//     one touched pheromone entry, tau' + the exact sum of its paths' weights
//     (Sec. 2.3, Eq. 3), formed the way the kernel forms it -- weights split
//     into 24-bit chunks in units of 2^E0 (E0 the smallest weight exponent;
//     two 27-bit chunks when every exponent is E0 or E0 + 1),
//     the chunks summed per word in any order, then rounded once;
//   - the tour length (csrc/exact_len.cuh, the tour-length kernel's code):
//     the edge lengths dealt to `groups` partial sums the way lanes and warps
//     take them, each partial sum normalised, the digit sums added, then
//     rounded once (Eq. 3).
#include <climits>

#include "exact.cuh"
#include "exact_len.cuh"

extern "C" {

// c: k >= 1 positive finite weights spanning at most kDepSpan binades.
// Writes fp32 bits (bf16 = 0) or the bfloat16 pattern (bf16 = 1) to *out;
// returns -1 if the weights are out of the fixed-point range.
int hx_deposit_entry(float tp, const double* c, int k, int bf16, uint32_t* out) {
  int e0 = INT_MAX, emax = INT_MIN;
  for (int i = 0; i < k; ++i) {
    const int e = aco::exponent_of(c[i]);
    e0 = e < e0 ? e : e0;
    emax = e > emax ? e : emax;
  }
  if (k < 1 || emax - e0 > aco::kDepSpan) return -1;
  uint64_t w0 = 0, w1 = 0, w2 = 0;
  const bool narrow = emax - e0 <= 1;  // as the kernel splits them: two 27-bit chunks, else three 24-bit
  for (int i = k - 1; i >= 0; --i) {  // any order: integer sums
    uint32_t a, b, d = 0;
    if (narrow)
      aco::weight_chunks27(c[i], e0, &a, &b);
    else
      aco::weight_chunks(c[i], e0, &a, &b, &d);
    w0 += a;
    w1 += b;
    w2 += d;
  }
  if (narrow) w1 <<= 3;
  *out = bf16 ? aco::round_sum_bf16(tp, w0, w1, w2, e0) : aco::bits_of(aco::round_sum_f32(tp, w0, w1, w2, e0));
  return 0;
}

int hx_dep_span() { return aco::kDepSpan; }

// Sum of count edge lengths split round-robin over `groups` partial sums, in
// reverse order within each group, each edge into the fast window or the
// full digits as the tour-length kernel adds it.  Returns -1 (and writes nothing) if an
// edge is outside the fixed-point range.
int hx_tour_length(const double* d, int count, int groups, double* out) {
  if (groups < 1) groups = 1;
  uint64_t total[aco::kLenDigits] = {};
  for (int g = 0; g < groups; ++g) {
    uint64_t acc[aco::kLenDigits] = {}, win[4] = {};
    for (int i = count - 1; i >= 0; --i) {
      if (i % groups != g) continue;
      const uint64_t b = aco::bits_of(d[i]);
      if (!aco::len_in_range(b)) return -1;
      if (!aco::len_win_add(win, b)) {  // as the kernel adds them: window, else its digits
        uint32_t w0, w1, w2;
        const int q = aco::len_digits(b, &w0, &w1, &w2);
        acc[q] += w0;
        acc[q + 1] += w1;
        acc[q + 2] += w2;
      }
    }
    uint64_t wd[5];
    aco::len_win_digits(win, wd);
    for (int i = 0; i < 5; ++i) acc[aco::kLenWin + i] += wd[i];
    aco::len_acc_carry(acc);
    for (int q = 0; q < aco::kLenDigits; ++q) total[q] += acc[q];
  }
  *out = aco::len_acc_round(total);
  return 0;
}
}
