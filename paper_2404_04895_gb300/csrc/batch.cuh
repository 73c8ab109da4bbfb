// Device-side description of one instance of a batch (many independent TSP
// instances advanced together by multi-instance kernels).
#pragma once

#include <stdint.h>

namespace aco {

struct InstDev {
  int n, m, ld, alpha;
  int adair, n_sched;
  int rw;                         // roulette-wheel construction (Sec. 2.4) instead of IR / AdaIR
  int topk;                       // paths that deposit (0: all)
  float rho, Q;
  uint2 key;                      // Philox key (seed low, high)
  const float* H;                 // eta^beta, n x ld
  float* tau;                     // n x ld, fp32 (tau_bf16: bf16 bit patterns, n x ld x 2 bytes)
  int tau_bf16;                   // M_tau stored in bfloat16
  void* P;                        // M_p, n x ld at the batch precision
  const double* D;                // strictly upper triangle, tri_index
  int32_t* tours;                 // m x n
  double* L;                      // m
  double* c;                      // m
  int2* dep;                      // deposit weights' scaling (E0, mode), written by best
  int32_t* nbr;                   // n x m x 2
  int32_t* best_tour;             // n
  double* best_len;               // 1
  uint32_t* it;                   // iterations completed (device counter)
  const float* sched;             // AdaIR 1/gamma per iteration (n_sched entries)
  uint2* lists;                   // candidate lists, n x kListMax (nullptr: full scan only, or rw)
  int* lcnt;                      // n
  uint32_t* lkey;                 // n
};

// Index of the instance whose half-open range [off[i], off[i+1]) holds x
// (off: exclusive prefix sums, off[count] = total).
__device__ __forceinline__ int find_instance(const int* __restrict__ off, int count, int x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

}  // namespace aco
