// Per-row / per-ant / per-instance device functions of the iteration steps
// other than tour construction.  The single-instance kernels (kernels.cu) and
// the multi-instance kernels (batch.cu) are thin wrappers around them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>

#include "common.cuh"
#include "exact.cuh"
#include "exact_len.cuh"
#include "lists.cuh"

namespace aco {

// ---------------------------------------------------------------------------
// Eq. 1 (unnormalised): X_ij = fl32(powi(tau_ij, alpha) * H_ij), X_ii = 0,
// AdaIR X_ij <- pow_own(X_ij, inv_gamma); FP16 rows scaled by 2^-e_i first.
// One row per call, all threads of the CTA, 4 columns per thread step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float p_entry(float tau, float h, int i, int j, int n, int alpha,
                                         float inv_gamma) {
  if (j >= n || j == i) return 0.0f;
  float x = __fmul_rn(powi_f32(tau, alpha), h);
  if (inv_gamma != 1.0f) x = pow_own(x, inv_gamma);
  return x;
}

// Entry (a, b), a < b, of the strictly upper triangle of an n x n symmetric
// matrix stored row by row (row a holds columns a + 1 .. n - 1): the solvers'
// distance matrix, n (n - 1) / 2 fp64 values.  a (2n - a - 1) is always even.
__host__ __device__ __forceinline__ size_t tri_index(int n, int a, int b) {
  return (size_t)a * (size_t)(2 * n - a - 1) / 2 + (size_t)(b - a - 1);
}

// Columns 4q .. 4q+3 of a tau row stored in fp32 (TB false) or bfloat16 (TB
// true), widened to fp32 (exact).  COH: the row was written earlier by the
// same kernel, so it is read through the L2 (not the read-only path).
template <bool TB, bool COH = false>
__device__ __forceinline__ float4 load_tau4(const void* __restrict__ row, int q) {
  if (!TB)
    return COH ? __ldcg(reinterpret_cast<const float4*>(row) + q) : __ldg(reinterpret_cast<const float4*>(row) + q);
  const uint2 u = COH ? __ldcg(reinterpret_cast<const uint2*>(row) + q) : __ldg(reinterpret_cast<const uint2*>(row) + q);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
}

template <int PREC, bool TB = false>
__device__ __forceinline__ void build_P_row(const void* __restrict__ tau_row,
                                            const float* __restrict__ H_row, int n, int ld, int i,
                                            int alpha, float inv_gamma, void* __restrict__ P_row,
                                            float* red /* [32] shared */) {
  const float4* h4 = reinterpret_cast<const float4*>(H_row);
  const int nq = ld >> 2;
  float scale = 1.0f;
  if (PREC == ACO_FP16) {
    float mx = 0.0f;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const float4 a = load_tau4<TB>(tau_row, q), b = __ldg(h4 + q);
      const int j = 4 * q;
      mx = fmaxf(mx, p_entry(a.x, b.x, i, j, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.y, b.y, i, j + 1, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.z, b.z, i, j + 2, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.w, b.w, i, j + 3, n, alpha, inv_gamma));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(ACO_FULL_MASK, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    __syncthreads();  // red may be reused by the caller's next row
    int e = 0;
    if (mx > 0.0f) {
      const int ef = (int)((__float_as_uint(mx) >> 23) & 0xFF);
      e = (ef == 0 ? -127 : ef - 127) - 14;
      e = e < -126 ? -126 : (e > 113 ? 113 : e);
    }
    scale = __uint_as_float((uint32_t)(127 - e) << 23);
  }
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const float4 a = load_tau4<TB>(tau_row, q), b = __ldg(h4 + q);
    const int j = 4 * q;
    const float x0 = p_entry(a.x, b.x, i, j, n, alpha, inv_gamma);
    const float x1 = p_entry(a.y, b.y, i, j + 1, n, alpha, inv_gamma);
    const float x2 = p_entry(a.z, b.z, i, j + 2, n, alpha, inv_gamma);
    const float x3 = p_entry(a.w, b.w, i, j + 3, n, alpha, inv_gamma);
    if (PREC == ACO_FP32) {
      reinterpret_cast<float4*>(P_row)[q] = make_float4(x0, x1, x2, x3);
    } else if (PREC == ACO_BF16) {
      const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x0)) |
                          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x1)) << 16);
      const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x2)) |
                          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x3)) << 16);
      reinterpret_cast<uint2*>(P_row)[q] = make_uint2(lo, hi);
    } else {
      const uint32_t lo = (uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x0, scale))) |
                          ((uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x1, scale))) << 16);
      const uint32_t hi = (uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x2, scale))) |
                          ((uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x3, scale))) << 16);
      reinterpret_cast<uint2*>(P_row)[q] = make_uint2(lo, hi);
    }
  }
}

// ---------------------------------------------------------------------------
// Eq. 3 + Eq. 2 for ant k, by W cooperating warps (w: this warp's index among
// them; all W warps of the CTA when W > 1).  f is the exact sum of the n fp64
// edge lengths D[p_t][p_{t+1 mod n}] rounded once (exact_len.cuh): lane l of
// warp w takes edges t = 32 w + l + 32 W i, four in flight at a time, and
// adds each to its four-digit fast window in registers, or, if the edge does
// not fit it, to the ant's eleven shared digits (atomics); the windows are
// summed over lanes (redux on 16-bit halves) and added to the shared digits
// by each warp -- integer sums, so the split changes no bit.  For city
// a = p_t the index mapping nbr[a][k] = (p_{t-1}, p_{t+1}); L_k and
// c_k = Q / L_k.  A tour with an edge length outside the fixed-point range
// (impossible for distances of fp32 coordinates) gets L_k = c_k = NaN.
// The index-mapping entry of city a goes to element a * nbs of nb (nb null:
// none): an int2 in global memory, or with PACK16 (n <= 65535) one 32-bit
// word (pred | succ << 16) of a shared staging area.  sacc: kLenDigits + 1
// shared words for this ant (one area per warp when W == 1, per W-warp group
// when W > 1).  W > 1: every warp of the CTA calls this (its block barriers).
// PACKED: D holds the strictly upper triangle (tri_index), else all n x n.
// ---------------------------------------------------------------------------
template <int W, bool PACK16 = false, bool PACKED = false>
__device__ __forceinline__ void tour_length_exact(const double* __restrict__ D, int n,
                                                  const int32_t* __restrict__ p, int k,
                                                  float Q, double* __restrict__ L,
                                                  double* __restrict__ c,
                                                  void* nb, int nbs, int w,
                                                  unsigned long long* sacc) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  if (32 * w + lane <= kLenDigits) sacc[32 * w + lane] = 0ull;
  if (W == 1)
    __syncwarp();
  else
    __syncthreads();
  uint64_t win[4] = {0ull, 0ull, 0ull, 0ull};
  bool bad = false;
  for (int t0 = 32 * w + lane; t0 < n; t0 += U * 32 * W) {
    uint64_t db[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * 32 * W;
      db[u] = 0ull;
      if (t < n) {
        const int cur = __ldg(p + t);
        const int nx = __ldg(p + (t + 1 < n ? t + 1 : 0));
        // tours come from the construction kernel; an entry out of range
        // (only after a failed construction, which the host reports) is skipped
        if ((unsigned)cur < (unsigned)n && (unsigned)nx < (unsigned)n) {
          if (!PACKED)
            db[u] = (uint64_t)__double_as_longlong(__ldg(D + (size_t)cur * n + nx));
          else if (cur != nx)  // d(a, a) = 0 (only a repeated city gives such an edge)
            db[u] = (uint64_t)__double_as_longlong(
                __ldg(D + (cur < nx ? tri_index(n, cur, nx) : tri_index(n, nx, cur))));
          if (nb) {
            const int pv = __ldg(p + (t > 0 ? t - 1 : n - 1));
            if (PACK16)
              static_cast<uint32_t*>(nb)[(size_t)cur * nbs] = ((uint32_t)pv & 0xFFFFu) | ((uint32_t)nx << 16);
            else
              static_cast<int2*>(nb)[(size_t)cur * nbs] = make_int2(pv, nx);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = len_in_range(db[u]);
      bad |= !ok;
      if (ok && !len_win_add(win, db[u])) {  // rare: an edge outside the window's binades
        uint32_t w0, w1, w2;
        const int q = len_digits(db[u], &w0, &w1, &w2);
        atomicAdd(sacc + q, (unsigned long long)w0);
        atomicAdd(sacc + q + 1, (unsigned long long)w1);
        atomicAdd(sacc + q + 2, (unsigned long long)w2);
      }
    }
  }
  uint64_t wd[5];
  len_win_digits(win, wd);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint32_t lo = __reduce_add_sync(ACO_FULL_MASK, (uint32_t)wd[i] & 0xFFFFu);
    const uint32_t hi = __reduce_add_sync(ACO_FULL_MASK, (uint32_t)(wd[i] >> 16));
    wd[i] = (uint64_t)lo + ((uint64_t)hi << 16);
  }
  bad = __any_sync(ACO_FULL_MASK, bad);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (wd[i]) atomicAdd(sacc + kLenWin + i, (unsigned long long)wd[i]);
    if (bad) atomicOr(sacc + kLenDigits, 1ull);
  }
  if (W == 1)
    __syncwarp();
  else
    __syncthreads();
  if (w != 0 || lane != 0) return;
  uint64_t acc[kLenDigits];
#pragma unroll
  for (int i = 0; i < kLenDigits; ++i) acc[i] = sacc[i];
  const double total = sacc[kLenDigits] ? __longlong_as_double(0x7FF8000000000000ll) : len_acc_round(acc);
  L[k] = total;
  if (c) c[k] = __ddiv_rn((double)Q, total);
}

// ---------------------------------------------------------------------------
// Iteration best (argmin L, lowest ant on ties) merged into the running best
// (strictly shorter only); all threads of the CTA.  Advances *it_dev, if given.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void best_block(const double* __restrict__ L,
                                           const int32_t* __restrict__ tours, int n, int m,
                                           int32_t* __restrict__ best_tour,
                                           double* __restrict__ best_len, uint32_t* it_dev,
                                           double* sl /* [32] shared */, int* sk /* [33] shared */) {
  double bl = INFINITY;
  int bk = 0x7FFFFFFF;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double v = L[k];
    if (v < bl || (v == bl && k < bk)) {
      bl = v;
      bk = k;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(ACO_FULL_MASK, bl, off);
    const int ok = __shfl_xor_sync(ACO_FULL_MASK, bk, off);
    if (ov < bl || (ov == bl && ok < bk)) {
      bl = ov;
      bk = ok;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sl[threadIdx.x >> 5] = bl;
    sk[threadIdx.x >> 5] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (sl[w] < bl || (sl[w] == bl && sk[w] < bk)) {
        bl = sl[w];
        bk = sk[w];
      }
    }
    const int take = (bk < m && bl < *best_len) ? 1 : 0;
    sk[32] = take ? bk : -1;
    if (take) *best_len = bl;
    if (it_dev) *it_dev = *it_dev + 1u;
  }
  __syncthreads();
  const int kb = sk[32];
  if (kb >= 0) {
    const int32_t* src = tours + (size_t)kb * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) best_tour[t] = src[t];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Sec. 2.3, selection of the deposit paths: the solution set sorted by
// length (ascending, equal lengths by ant index) and the first k kept.  The
// weight c_j of every other ant is set to 0, so it deposits nothing.  Radix
// select of the k-th smallest length (its fp64 bit pattern, order-preserving
// for lengths >= 0), 8 bits per pass from the top; the kept lengths equal to
// it are those of the lowest ant indices.  k <= 0 or k >= m keeps every ant.
// All threads of the CTA (blockDim.x a multiple of 32, <= 1024); sred: 300
// ints of shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void select_topk_block(const double* __restrict__ L, int m, int k,
                                                  double* __restrict__ c, int* sred) {
  if (k <= 0 || k >= m) return;
  uint32_t* hist = reinterpret_cast<uint32_t*>(sred);  // [256]
  int* sh = sred + 256;                                // [0..1] prefix, [2] need, [3] below, [8..39] warp sums
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long prefix = 0ull;
  uint32_t need = (uint32_t)k, below = 0u;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += nt) hist[b] = 0u;
    __syncthreads();
    const unsigned long long hi_mask = shift == 56 ? 0ull : (~0ull << (shift + 8));
    for (int j = tid; j < m; j += nt) {
      const unsigned long long key = (unsigned long long)__double_as_longlong(L[j]);
      if ((key & hi_mask) == prefix) atomicAdd(hist + (int)((key >> shift) & 0xFFull), 1u);
    }
    __syncthreads();
    if (wid == 0) {  // lane l holds bins 8l .. 8l+7 (ascending)
      uint32_t h[8], sum = 0u;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        h[i] = hist[8 * lane + i];
        sum += h[i];
      }
      uint32_t inc = sum;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(ACO_FULL_MASK, inc, off);
        if (lane >= off) inc += v;
      }
      uint32_t cum = inc - sum;
      if (cum < need && inc >= need) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (cum + h[i] >= need) {
            const unsigned long long px = prefix | ((unsigned long long)(8 * lane + i) << shift);
            sh[0] = (int)(uint32_t)px;
            sh[1] = (int)(uint32_t)(px >> 32);
            sh[2] = (int)(need - cum);
            sh[3] = (int)cum;
            break;
          }
          cum += h[i];
        }
      }
    }
    __syncthreads();
    prefix = (unsigned long long)(uint32_t)sh[0] | ((unsigned long long)(uint32_t)sh[1] << 32);
    need = (uint32_t)sh[2];
    below += (uint32_t)sh[3];
    __syncthreads();
  }
  // keep: key < T, or key == T among the first `need` such ants by index;
  // each thread takes a contiguous run of ants, ranks by an exclusive scan
  const unsigned long long T = prefix;
  const int span = (m + nt - 1) / nt;
  const int j0 = tid * span, j1 = min(m, j0 + span);
  uint32_t my_eq = 0u;
  for (int j = j0; j < j1; ++j) my_eq += (unsigned long long)__double_as_longlong(L[j]) == T;
  uint32_t inc = my_eq;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(ACO_FULL_MASK, inc, off);
    if (lane >= off) inc += v;
  }
  if (lane == 31) sh[8 + wid] = (int)inc;
  __syncthreads();
  uint32_t rank = inc - my_eq;
  for (int w = 0; w < wid; ++w) rank += (uint32_t)sh[8 + w];
  for (int j = j0; j < j1; ++j) {
    const unsigned long long key = (unsigned long long)__double_as_longlong(L[j]);
    bool keep = key < T;
    if (key == T) keep = rank++ < need;
    if (!keep) c[j] = 0.0;
  }
  __threadfence_block();
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Scaling of the deposit weights c[0..m) for the exact fixed-point sums
// (exact.cuh): x = E0, the smallest exponent of a positive finite weight, and
// y = mode: kDepNarrow if every weight's exponent is E0 or E0 + 1 (two
// 27-bit chunks each), else kDepFixed; kDepInf if some weight is +inf (a zero tour length:
// every city at one point); kDepBad if a weight is negative or NaN, or the
// positive ones span more than kDepSpan binades (tour lengths of one planar
// instance span at most log2(n) + 1).  All threads of the CTA; every thread
// gets the result.  sred: 100 ints of shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int2 deposit_scale_block(const double* __restrict__ c, int m, int* sred) {
  int emin = INT_MAX, emax = INT_MIN;
  unsigned flags = 0u;  // 1: +inf seen, 2: negative or NaN seen
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double v = c[k];
    if (v > 0.0 && v < INFINITY) {
      const int e = exponent_of(v);
      emin = min(emin, e);
      emax = max(emax, e);
    } else if (v == INFINITY) {
      flags |= 1u;
    } else if (!(v == 0.0)) {
      flags |= 2u;
    }
  }
  emin = __reduce_min_sync(ACO_FULL_MASK, emin);
  emax = __reduce_max_sync(ACO_FULL_MASK, emax);
  flags = __reduce_or_sync(ACO_FULL_MASK, flags);
  const int w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  if ((threadIdx.x & 31) == 0) {
    sred[w] = emin;
    sred[32 + w] = emax;
    sred[64 + w] = (int)flags;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    const int a = __reduce_min_sync(ACO_FULL_MASK, l < nw ? sred[l] : INT_MAX);
    const int b = __reduce_max_sync(ACO_FULL_MASK, l < nw ? sred[32 + l] : INT_MIN);
    const unsigned f = __reduce_or_sync(ACO_FULL_MASK, l < nw ? (unsigned)sred[64 + l] : 0u);
    if (l == 0) {
      sred[96] = a;
      sred[97] = b;
      sred[98] = (int)f;
    }
  }
  __syncthreads();
  emin = sred[96];
  emax = sred[97];
  flags = (unsigned)sred[98];
  __syncthreads();  // sred may be reused by the caller
  int mode = (flags & 2u) ? kDepBad : (flags & 1u) ? kDepInf : kDepFixed;
  if (emin != INT_MAX && emax - emin > kDepSpan) mode = kDepBad;
  if (mode == kDepFixed && emin != INT_MAX && emax - emin <= 1) mode = kDepNarrow;
  return make_int2(emin == INT_MAX ? 0 : emin, mode);
}

// ---------------------------------------------------------------------------
// Sec. 2.3 evaporation + deposit of one row a (all threads of the CTA), in
// the order-free reading: tau'_ab = fl32(keep * tau_ab) with keep =
// fl32(1 - rho); an entry that some path uses becomes tau'_ab + the sum of
// those paths' weights, taken exactly and rounded once to fp32.
//   1. the row's 2m index-mapping entries (two neighbours per ant) mark the
//      touched columns in a shared bitmap
//   2. a touched column's slot is the number of touched columns before it
//      (exclusive scan of the bitmap's popcounts), so slots are dense
//   3. each warp takes 32 ants at a time: lanes whose columns share a slot
//      are grouped by __match_any_sync, their 24-bit weight chunks summed by
//      one redux per chunk, and the group's leader adds the sums to the
//      slot's carry-save words with shared atomics (integer sums: any order
//      gives the same bits)
//   4. one thread per slot rounds tau' + its sum once (into a shared table),
//      then one coalesced pass over the row writes tau' or the slot's result
// At most `cap` slots are summed per pass; rows with more touched columns
// take further passes (only their touched columns are rewritten).  With
// weights the fixed point cannot hold (mode kDepBad: a weight negative or NaN,
// or the positive ones spanning more than kDepSpan binades) every touched
// entry becomes NaN and the others tau'.
// smem: deposit_smem_bytes(n, cap).
// ---------------------------------------------------------------------------
// w += v for a 64-bit shared word w kept as two 32-bit halves (w[0] low):
// one 32-bit atomic add, and a second on the high half only when the low one
// wraps -- every carry is counted once whatever the interleaving, and shared
// 32-bit atomics run several times faster than 64-bit ones on this GPU.
__device__ __forceinline__ void dep_add_u64(uint32_t* w, uint32_t v) {
  const uint32_t old = atomicAdd(w, v);
  if (old + v < old) atomicAdd(w + 1, 1u);
}

constexpr int kDepThreads = 256;
constexpr int kDepCap = 512;  // 16 KB of slots: a row's touched columns are few once tours share edges

__host__ __device__ inline int deposit_cap(int n, long long m) {
  long long c = 2 * m < (long long)n ? 2 * m : (long long)n;
  return (int)(c < kDepCap ? c : kDepCap);
}

__host__ __device__ inline size_t deposit_smem_bytes(int n, int cap) {
  const size_t nw = (size_t)(n + 31) / 32;
  return (size_t)cap * 32 + nw * 8 + 33 * 4 + (size_t)cap * 8;
}

template <bool TB = false>
__device__ __forceinline__ void deposit_row_exact(void* __restrict__ row_v, int n,
                                                  const int2* __restrict__ nbr_row,
                                                  const double* __restrict__ c, int m, float keep,
                                                  int E0, int mode, int cap, unsigned char* smem) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x;
  const int nw = (n + 31) >> 5;
  // [cap][4]: per slot the carry-save words w0, w1, w2 (each as two 32-bit
  // halves, see dep_add_u64) and the count of infinite weights
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* bm = reinterpret_cast<uint32_t*>(acc + (size_t)cap * 4);      // [nw]
  uint32_t* base = bm + nw;                                                // [nw]
  int* sc = reinterpret_cast<int*>(base + nw);                             // [33]
  int* tcol = sc + 33;                                                     // [cap] column of each slot of a pass
  uint32_t* res = reinterpret_cast<uint32_t*>(tcol + cap);                 // [cap] its rounded result

  // 1. touched columns
  for (int w = tid; w < nw; w += nthr) bm[w] = 0u;
  __syncthreads();
  // a bit already seen set needs no atomic (a stale read only repeats one);
  // ants of weight 0 (not selected) leave their entries at tau'
  for (int k = tid; k < m; k += nthr) {
    if (__ldg(c + k) == 0.0) continue;
    const int2 e = __ldg(nbr_row + k);
    if ((unsigned)e.x < (unsigned)n && !((bm[e.x >> 5] >> (e.x & 31)) & 1u))
      atomicOr(bm + (e.x >> 5), 1u << (e.x & 31));
    if ((unsigned)e.y < (unsigned)n && !((bm[e.y >> 5] >> (e.y & 31)) & 1u))
      atomicOr(bm + (e.y >> 5), 1u << (e.y & 31));
  }
  __syncthreads();

  // 2. dense slots: exclusive scan of the popcounts, each thread a run of words
  const int per = (nw + nthr - 1) / nthr;
  const int wb = tid * per;
  int loc = 0;
  for (int q = 0; q < per; ++q)
    if (wb + q < nw) loc += __popc(bm[wb + q]);
  int incl = loc;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(ACO_FULL_MASK, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) sc[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int v = lane < (nthr >> 5) ? sc[lane] : 0;
    int inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(ACO_FULL_MASK, inc, off);
      if (lane >= off) inc += u;
    }
    sc[lane] = inc - v;
    if (lane == 31) sc[32] = inc;
  }
  __syncthreads();
  {
    int run = sc[warp] + incl - loc;
    for (int q = 0; q < per; ++q)
      if (wb + q < nw) {
        base[wb + q] = (uint32_t)run;
        run += __popc(bm[wb + q]);
      }
  }
  const int D = sc[32];
  __syncthreads();
  auto slot_of = [&](int j) -> int {
    return (int)base[j >> 5] + __popc(bm[j >> 5] & ((1u << (j & 31)) - 1u));
  };

  float* row = static_cast<float*>(row_v);                // fp32 storage
  unsigned short* rowh = static_cast<unsigned short*>(row_v);  // bf16 storage
  // weights the fixed point cannot hold (mode kDepBad): one pass that writes
  // NaN to every touched entry, so the failure shows in tau itself
  const int npass = D > 0 && mode != kDepBad ? (D + cap - 1) / cap : 1;
  for (int p = 0; p < npass; ++p) {
    const int s0 = p * cap;
    const int used = min(cap, D - s0);
    for (int q = tid; q < used * 4; q += nthr) acc[q] = 0ull;
    __syncthreads();

    // 3. exact sums
    if (used > 0 && mode != kDepBad) {
      for (int kb = warp * 32; kb < m; kb += nthr) {
        const int k = kb + lane;
        const bool valid = k < m;
        int2 e = make_int2(-1, -1);
        uint32_t q0 = 0u, q1 = 0u, q2 = 0u, qi = 0u;
        if (valid) {
          e = __ldg(nbr_row + k);
          const double v = __ldg(c + k);
          if (v > 0.0 && v < INFINITY) {
            if (mode == kDepNarrow)
              weight_chunks27(v, E0, &q0, &q1);
            else
              weight_chunks(v, E0, &q0, &q1, &q2);
          } else if (v == INFINITY)
            qi = 1u;
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int col = side ? e.y : e.x;
          const bool ok = valid && (unsigned)col < (unsigned)n;
          const int sl = ok ? slot_of(col) - s0 : -1;
          const bool in = ok && sl >= 0 && sl < cap;
          const unsigned grp = __match_any_sync(ACO_FULL_MASK, in ? sl : -1 - lane);
          const uint32_t r0 = __reduce_add_sync(grp, in ? q0 : 0u);
          const uint32_t r1 = __reduce_add_sync(grp, in ? q1 : 0u);
          uint32_t r2 = 0u;  // (no third chunk in the narrow form)
          if (mode != kDepNarrow) r2 = __reduce_add_sync(grp, in ? q2 : 0u);
          uint32_t ri = 0u;
          if (mode == kDepInf) ri = __reduce_add_sync(grp, in ? qi : 0u);
          if (in && lane == __ffs(grp) - 1) {
            uint32_t* a = reinterpret_cast<uint32_t*>(acc + 4 * sl);
            if (r0) dep_add_u64(a + 0, r0);
            if (r1) dep_add_u64(a + 2, r1);
            if (r2) dep_add_u64(a + 4, r2);
            if (ri) atomicAdd(a + 6, ri);
          }
        }
      }
    }
    __syncthreads();

    // 4a. each slot of this pass: its column (from the bitmap), then tau' +
    //     the slot's sum rounded once, from the entry's stored value (not yet
    //     rewritten: the row pass below and later passes leave it alone
    //     until then); stored in fp32, or in bf16 (to nearest even)
    if (used > 0 && mode != kDepBad) {
      for (int q = 0; q < per; ++q) {
        const int w = wb + q;
        if (w >= nw) break;
        uint32_t bits = bm[w];
        int sl = (int)base[w] - s0;
        while (bits) {
          if (sl >= used) break;
          const int b = __ffs(bits) - 1;
          bits &= bits - 1u;
          if (sl >= 0) tcol[sl] = 32 * w + b;
          ++sl;
        }
      }
      __syncthreads();
      for (int sl = tid; sl < used; sl += nthr) {
        const int j = tcol[sl];
        const float tp = __fmul_rn(keep, TB ? __uint_as_float((uint32_t)rowh[j] << 16) : row[j]);
        const uint32_t* a = reinterpret_cast<const uint32_t*>(acc + 4 * sl);
        const uint64_t w0 = ((uint64_t)a[1] << 32) | a[0], w2 = ((uint64_t)a[5] << 32) | a[4];
        uint64_t w1 = ((uint64_t)a[3] << 32) | a[2];
        if (mode == kDepNarrow) w1 <<= 3;  // units of 2^27 -> 2^24 (w1 < 2m 2^27 <= 2^48)
        if (mode == kDepInf && a[6])
          res[sl] = TB ? 0x7F80u : 0x7F800000u;
        else
          res[sl] = TB ? round_sum_bf16(tp, w0, w1, w2, E0) : __float_as_uint(round_sum_f32(tp, w0, w1, w2, E0));
      }
      __syncthreads();
    }

    // 4b. the row: tau' everywhere on the first pass, each touched entry's
    //     result from its slot
    for (int q = tid; 4 * q < n; q += nthr) {
      const int j0 = 4 * q;
      const uint32_t nib = (bm[j0 >> 5] >> (j0 & 31)) & 0xFu;
      if (p > 0 && nib == 0u) continue;
      const bool full = j0 + 4 <= n;
      float v[4];
      if (full) {
        const float4 x = load_tau4<TB>(row_v, q);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          v[i] = j0 + i < n ? (TB ? __uint_as_float((uint32_t)rowh[j0 + i] << 16) : row[j0 + i]) : 0.0f;
      }
      uint32_t out[4];  // fp32 bits, or bf16 bits in the low half
      bool write[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float tp = __fmul_rn(keep, v[i]);
        write[i] = true;
        if (!((nib >> i) & 1u)) {
          if (p == 0) {
            out[i] = TB ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(tp)) : __float_as_uint(tp);
          } else {
            write[i] = false;
          }
          continue;
        }
        if (mode == kDepBad) {
          out[i] = TB ? 0x7FC0u : 0x7FC00000u;
          continue;
        }
        const int sl = slot_of(j0 + i) - s0;
        if (sl < 0 || sl >= cap) {  // summed in another pass
          write[i] = false;
          continue;
        }
        out[i] = res[sl];
      }
      // entries not written in this pass keep their stored bits
      if (full && write[0] && write[1] && write[2] && write[3]) {
        if (TB)
          reinterpret_cast<uint2*>(row_v)[q] = make_uint2(out[0] | (out[1] << 16), out[2] | (out[3] << 16));
        else
          reinterpret_cast<uint4*>(row_v)[q] = make_uint4(out[0], out[1], out[2], out[3]);
      } else {
        for (int i = 0; i < 4 && j0 + i < n; ++i)
          if (write[i]) {
            if (TB)
              rowh[j0 + i] = (unsigned short)out[i];
            else
              row[j0 + i] = __uint_as_float(out[i]);
          }
      }
    }
    __syncthreads();
  }
}

}  // namespace aco

namespace aco {

// ---------------------------------------------------------------------------
// Candidate list of row i of M_p (exact fast path of the construction step).
// Keys are the fp32 bit patterns of the stored values (>= 0, so key order is
// value order).  With T the kListTarget-th largest key of the row (radix
// select, 8 bits per pass), the list holds every column with key > T and
// columns with key == T up to kListMax entries, sorted by key (descending,
// ties by column); bkey bounds the score key (fp32 bits + 1, see construct)
// of every column left out:
//   all columns with key >= T listed  ->  outside keys < T,  bkey = T
//   ties at T truncated               ->  outside keys <= T, bkey = T + 1
//   row has <= kListMax columns        ->  nothing outside,   bkey = 0
// Sorted, the first r entries bound the rest: a column after them has a
// score key <= key(entry r) + 1.  A step is decided by the list when its best
// score over the entries scored so far exceeds the bound of everything else:
// no other column can then reach (or tie) that score.
// Slots past the count are written as (0, kListPad), so a reader can tell a
// listed entry from its own slot.  All threads of the CTA (blockDim.x <= 256);
// scratch: kListScratchWords shared words.
// ---------------------------------------------------------------------------
constexpr int kListScratchWords = 256 + 8 + 2 * kListMax * 2;

// COH: the row was written by the same kernel (read through the L2 with
// ordinary loads, not the read-only path)
template <int PREC, bool COH = false>
__device__ __forceinline__ uint32_t p_key(const void* __restrict__ row, int j) {
  if (PREC == ACO_FP32)
    return COH ? __ldcg(static_cast<const uint32_t*>(row) + j) : __ldg(static_cast<const uint32_t*>(row) + j);
  const uint32_t h = COH ? __ldcg(static_cast<const unsigned short*>(row) + j)
                         : __ldg(static_cast<const unsigned short*>(row) + j);
  if (PREC == ACO_BF16) return h << 16;
  return __float_as_uint(__half2float(__ushort_as_half((unsigned short)h)));
}

// Keys (fp32 bit patterns) of the KV columns of 16-byte chunk q of a row.
template <int PREC, bool COH = false>
struct RowKeys {
  static constexpr int KV = PREC == ACO_FP32 ? 4 : 8;
  uint32_t k[KV];
  __device__ __forceinline__ void load(const void* __restrict__ row, int q) {
    const uint4 d = COH ? __ldcg(static_cast<const uint4*>(row) + q) : __ldg(static_cast<const uint4*>(row) + q);
    if (PREC == ACO_FP32) {
      k[0] = d.x;
      k[1] = d.y;
      k[2] = d.z;
      k[3] = d.w;
    } else {
      const uint32_t w[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (PREC == ACO_BF16) {
          k[2 * i] = w[i] << 16;
          k[2 * i + 1] = w[i] & 0xFFFF0000u;
        } else {
          k[2 * i] = __float_as_uint(__half2float(__ushort_as_half((unsigned short)(w[i] & 0xFFFFu))));
          k[2 * i + 1] = __float_as_uint(__half2float(__ushort_as_half((unsigned short)(w[i] >> 16))));
        }
      }
    }
  }
};

// Bitonic sort, descending, of the first S (a power of two, <= 2 * blockDim.x)
// 64-bit keys of sk; all threads of the CTA.  Strides are powers of two, so
// a thread's pair index is formed with masks and a shift (no division).
__device__ __forceinline__ void bitonic_desc(unsigned long long* sk, int S) {
  const int tid = threadIdx.x;
  for (int size = 2; size <= S; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (tid < S / 2) {
        const int i = ((tid & ~(stride - 1)) << 1) | (tid & (stride - 1));  // 2*stride*(tid/stride) + tid%stride
        const int partner = i + stride;
        const bool desc = (i & size) == 0;
        const unsigned long long a = sk[i], b = sk[partner];
        if (desc ? (a < b) : (a > b)) {
          sk[i] = b;
          sk[partner] = a;
        }
      }
      __syncthreads();
    }
  }
}

// The same network as bitonic_desc(sk, 512), for a CTA of exactly 256
// threads and mostly in registers: thread t = 32w + l holds elements e =
// 64w + 2l and e + 1, so a partner at distance 1 is the thread's other
// element, one at distance 2..32 the same element of lane l ^ (d / 2) (a
// shuffle), and only distances >= 64 (6 of the 45 stages) go through sk with
// a barrier each.  Ends with sk sorted and a barrier.
__device__ __forceinline__ void bitonic512_desc_cta(unsigned long long* sk) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int e0 = ((tid >> 5) << 6) | (lane << 1);
  unsigned long long v0 = sk[e0], v1 = sk[e0 + 1];
#pragma unroll
  for (int size = 2; size <= 512; size <<= 1) {
    const bool desc = (e0 & size) == 0;  // the same for e0 + 1 (size >= 2)
    int stride = size >> 1;
    if (stride >= 64) {
      sk[e0] = v0;
      sk[e0 + 1] = v1;
      __syncthreads();
#pragma unroll
      for (; stride >= 64; stride >>= 1) {
        const int i = ((tid & ~(stride - 1)) << 1) | (tid & (stride - 1));
        const bool d = (i & size) == 0;
        const unsigned long long a = sk[i], b = sk[i + stride];
        if (d ? (a < b) : (a > b)) {
          sk[i] = b;
          sk[i + stride] = a;
        }
        __syncthreads();
      }
      v0 = sk[e0];  // each thread reloads (and later stores) only its own two
      v1 = sk[e0 + 1];
    }
#pragma unroll
    for (; stride >= 2; stride >>= 1) {
      const int ld = stride >> 1;
      const bool keep_max = ((lane & ld) == 0) == desc;  // lower element of a descending pair, or upper of an ascending
      const unsigned long long o0 = __shfl_xor_sync(ACO_FULL_MASK, v0, ld);
      const unsigned long long o1 = __shfl_xor_sync(ACO_FULL_MASK, v1, ld);
      v0 = (keep_max == (v0 > o0)) ? v0 : o0;
      v1 = (keep_max == (v1 > o1)) ? v1 : o1;
    }
    const bool gt = v0 > v1;
    const unsigned long long hi = gt ? v0 : v1, lo = gt ? v1 : v0;
    v0 = desc ? hi : lo;
    v1 = desc ? lo : hi;
  }
  sk[e0] = v0;
  sk[e0 + 1] = v1;
  __syncthreads();
}

// composite sort key: value bits high, complemented column low (ties: lower column first)
__device__ __forceinline__ unsigned long long list_sort_key(uint32_t key, int j) {
  return ((unsigned long long)key << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)j);
}

template <int PREC, bool COH = false>
__device__ __forceinline__ void build_list_row(const void* __restrict__ P_row, int n,
                                               uint2* __restrict__ list, int* __restrict__ cnt_out,
                                               uint32_t* __restrict__ bkey_out,
                                               uint32_t* scratch) {
  using RK = RowKeys<PREC, COH>;
  constexpr int KV = RK::KV;
  uint32_t* hist = scratch;                 // [256]
  uint32_t* sh = scratch + 256;             // [0] prefix [1] need [2] above [3] count [4] eq
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(scratch + 256 + 8);  // [kListMax]
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int nq = (n + KV - 1) / KV;  // 16-byte chunks (rows are padded to a multiple of 8)
  int S = 2;

  if (n <= kListMax) {  // every column listed, bound 0
    while (S < n) S <<= 1;
    for (int q = tid; q < S; q += nt) sk[q] = q < n ? list_sort_key(p_key<PREC, COH>(P_row, q), q) : 0ull;
    if (tid == 0) {
      *cnt_out = n;
      *bkey_out = 0u;
    }
    __syncthreads();
  } else {
    // 1. radix select of the kListTarget-th largest key T, 8 bits per pass from
    //    the top; keys above the chosen digit of a pass are above T, so their
    //    counts add up to the number of keys > T
    uint32_t prefix = 0u, need = kListTarget, above = 0u, n_eq = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
      for (int b = tid; b < 256; b += nt) hist[b] = 0u;
      __syncthreads();
      const uint32_t hi_mask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
      for (int q = tid; q < nq; q += nt) {
        RK r;
        r.load(P_row, q);
#pragma unroll
        for (int i = 0; i < KV; ++i)
          if (q < nq && q * KV + i < n && (r.k[i] & hi_mask) == prefix) atomicAdd(hist + ((r.k[i] >> shift) & 0xFFu), 1u);
      }
      __syncthreads();
      if (wid == 0) {
        // lane l holds bins 255-8l .. 248-8l (descending); exclusive prefix of
        // the lane sums from the top, then the lane whose run crosses `need`
        uint32_t h[8], sum = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          h[i] = hist[255 - 8 * lane - i];
          sum += h[i];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t v = __shfl_up_sync(ACO_FULL_MASK, inc, off);
          if (lane >= off) inc += v;
        }
        uint32_t cum = inc - sum;
        if (cum < need && inc >= need) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (cum + h[i] >= need) {
              sh[0] = prefix | ((uint32_t)(255 - 8 * lane - i) << shift);
              sh[1] = need - cum;
              sh[2] = cum;
              sh[4] = h[i];
              break;
            }
            cum += h[i];
          }
        }
      }
      __syncthreads();
      prefix = sh[0];
      need = sh[1];
      above += sh[2];
      n_eq = sh[4];
      __syncthreads();  // sh is rewritten by the next pass
    }
    const uint32_t T = prefix;
    const uint32_t n_gt = above;
    const bool all_ties = n_gt + n_eq <= (uint32_t)kListMax;
    const uint32_t eq_take = all_ties ? n_eq : (uint32_t)kListMax - n_gt;
    const int cnt = (int)(n_gt + eq_take);
    // 2. compaction into sk in any order (the sort restores it), except that
    //    when ties at T are cut the kept ones are the lowest columns
    if (tid == 0) sh[3] = 0u;
    __syncthreads();
    for (int q = tid; q < nq; q += nt) {
      RK r;
      r.load(P_row, q);
#pragma unroll
      for (int i = 0; i < KV; ++i) {
        const int j = q * KV + i;
        if (j < n && (r.k[i] > T || (all_ties && r.k[i] == T))) sk[atomicAdd(sh + 3, 1u)] = list_sort_key(r.k[i], j);
      }
    }
    if (!all_ties) {
      // the first eq_take columns equal to T, in column order: each thread
      // takes a contiguous span of columns
      const int span = (n + nt - 1) / nt;
      const int j0 = tid * span, j1 = min(n, j0 + span);
      uint32_t my_eq = 0u;
      for (int j = j0; j < j1; ++j) my_eq += p_key<PREC, COH>(P_row, j) == T;
      uint32_t inc = my_eq;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(ACO_FULL_MASK, inc, off);
        if (lane >= off) inc += v;
      }
      __syncthreads();
      if (lane == 31) hist[wid] = inc;  // warp totals (hist is free again)
      __syncthreads();
      uint32_t rank = inc - my_eq;
      for (int w = 0; w < wid; ++w) rank += hist[w];
      for (int j = j0; j < j1 && rank < eq_take; ++j)
        if (p_key<PREC, COH>(P_row, j) == T) sk[n_gt + rank++] = list_sort_key(T, j);
    }
    while (S < cnt) S <<= 1;
    __syncthreads();
    for (int q = cnt + tid; q < S; q += nt) sk[q] = 0ull;  // padding sorts last
    if (tid == 0) {
      *cnt_out = cnt;
      *bkey_out = all_ties ? T : T + 1u;
    }
    __syncthreads();
  }
  // 3. sort by key descending (ties: lower column first); write every slot
  bitonic_desc(sk, S);
  for (int q = tid; q < kListMax; q += nt) {
    const unsigned long long v = q < S ? sk[q] : 0ull;
    list[q] = v ? make_uint2((uint32_t)(v >> 32), 0xFFFFFFFFu - (uint32_t)v) : make_uint2(0u, kListPad);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Eq. 1 and the candidate list of the same row in one pass (solvers and
// batches): the row of M_p is computed and stored exactly as build_P_row
// does, and every column whose stored value's key reaches `guess` is
// collected on the way (at most kListMax).  If between kListTarget and
// kListMax columns reached it, they include every column whose key is >= T,
// the kListTarget-th largest key (at least kListTarget keys are >= guess, so
// T >= guess): sorted, they give T, and the list and bound of
// build_list_row's definition -- every key >= T then fits, so nothing is
// cut and the bound is T.  Any other count (a guess too high or too low, or
// none) falls back to build_list_row's radix select on the stored row.  The
// result is the same either way; the guess only decides the cost.
// guess: 0xFFFFFFFF for none.  scratch: kListScratchWords shared words plus
// `red` (32 floats) for the FP16 row maximum.  COH: the tau row was written
// earlier by the same kernel (load_tau4).
// ---------------------------------------------------------------------------
template <int PREC, bool TB = false, bool COH = false>
__device__ __forceinline__ void build_P_lists_row(const void* __restrict__ tau_row, const float* __restrict__ H_row,
                                                  int n, int ld, int i, int alpha, float inv_gamma,
                                                  void* __restrict__ P_row, uint2* __restrict__ list,
                                                  int* __restrict__ cnt_out, uint32_t* __restrict__ bkey_out,
                                                  uint32_t guess, uint32_t* scratch, float* red) {
  const float4* h4 = reinterpret_cast<const float4*>(H_row);
  const int nq = ld >> 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  uint32_t* sh = scratch + 256;
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(scratch + 256 + 8);
  if (n <= kListMax) guess = 0u;  // every column is listed: collect them all
  float scale = 1.0f;
  if (PREC == ACO_FP16) {
    float mx = 0.0f;
    for (int q = tid; q < nq; q += nt) {
      const float4 a = load_tau4<TB, COH>(tau_row, q), b = __ldg(h4 + q);
      const int j = 4 * q;
      mx = fmaxf(mx, p_entry(a.x, b.x, i, j, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.y, b.y, i, j + 1, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.z, b.z, i, j + 2, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.w, b.w, i, j + 3, n, alpha, inv_gamma));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(ACO_FULL_MASK, mx, off));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(nt >> 5); ++w) mx = fmaxf(mx, red[w]);
    int e = 0;
    if (mx > 0.0f) {
      const int ef = (int)((__float_as_uint(mx) >> 23) & 0xFF);
      e = (ef == 0 ? -127 : ef - 127) - 14;
      e = e < -126 ? -126 : (e > 113 ? 113 : e);
    }
    scale = __uint_as_float((uint32_t)(127 - e) << 23);
  }
  if (tid == 0) sh[3] = 0u;
  __syncthreads();
  auto collect = [&](uint32_t key, int j) {
    if (j < n && key >= guess) {
      const uint32_t slot = atomicAdd(sh + 3, 1u);
      if (slot < (uint32_t)kListMax) sk[slot] = list_sort_key(key, j);
    }
  };
  for (int q = tid; q < nq; q += nt) {
    const float4 a = load_tau4<TB, COH>(tau_row, q), b = __ldg(h4 + q);
    const int j = 4 * q;
    const float x0 = p_entry(a.x, b.x, i, j, n, alpha, inv_gamma);
    const float x1 = p_entry(a.y, b.y, i, j + 1, n, alpha, inv_gamma);
    const float x2 = p_entry(a.z, b.z, i, j + 2, n, alpha, inv_gamma);
    const float x3 = p_entry(a.w, b.w, i, j + 3, n, alpha, inv_gamma);
    uint32_t k0, k1, k2, k3;
    if (PREC == ACO_FP32) {
      reinterpret_cast<float4*>(P_row)[q] = make_float4(x0, x1, x2, x3);
      k0 = __float_as_uint(x0);
      k1 = __float_as_uint(x1);
      k2 = __float_as_uint(x2);
      k3 = __float_as_uint(x3);
    } else if (PREC == ACO_BF16) {
      const uint32_t b0 = __bfloat16_as_ushort(__float2bfloat16_rn(x0)), b1 = __bfloat16_as_ushort(__float2bfloat16_rn(x1));
      const uint32_t b2 = __bfloat16_as_ushort(__float2bfloat16_rn(x2)), b3 = __bfloat16_as_ushort(__float2bfloat16_rn(x3));
      reinterpret_cast<uint2*>(P_row)[q] = make_uint2(b0 | (b1 << 16), b2 | (b3 << 16));
      k0 = b0 << 16;
      k1 = b1 << 16;
      k2 = b2 << 16;
      k3 = b3 << 16;
    } else {
      const __half h0 = __float2half_rn(__fmul_rn(x0, scale)), h1 = __float2half_rn(__fmul_rn(x1, scale));
      const __half h2 = __float2half_rn(__fmul_rn(x2, scale)), h3 = __float2half_rn(__fmul_rn(x3, scale));
      reinterpret_cast<uint2*>(P_row)[q] =
          make_uint2((uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16),
                     (uint32_t)__half_as_ushort(h2) | ((uint32_t)__half_as_ushort(h3) << 16));
      k0 = __float_as_uint(__half2float(h0));
      k1 = __float_as_uint(__half2float(h1));
      k2 = __float_as_uint(__half2float(h2));
      k3 = __float_as_uint(__half2float(h3));
    }
    collect(k0, j);
    collect(k1, j + 1);
    collect(k2, j + 2);
    collect(k3, j + 3);
  }
  __syncthreads();
  const uint32_t cnt = sh[3];
  const bool all = n <= kListMax;
  if (all || (cnt >= (uint32_t)kListTarget && cnt <= (uint32_t)kListMax)) {
    int S = 2;
    while (S < (int)cnt) S <<= 1;
    for (int q = (int)cnt + tid; q < S; q += nt) sk[q] = 0ull;  // padding sorts last
    __syncthreads();
    if (S == 512 && nt == 256)
      bitonic512_desc_cta(sk);
    else
      bitonic_desc(sk, S);
    // T and the number of collected keys >= T (all of them >= T when n <= kListMax)
    const uint32_t T = all ? 0u : (uint32_t)(sk[kListTarget - 1] >> 32);
    if (tid == 0) sh[5] = cnt;
    __syncthreads();
    for (int q = tid; q < (int)cnt; q += nt)
      if ((uint32_t)(sk[q] >> 32) >= T && (q + 1 == (int)cnt || (uint32_t)(sk[q + 1] >> 32) < T)) sh[5] = (uint32_t)(q + 1);
    __syncthreads();
    const int take = (int)sh[5];
    for (int q = tid; q < kListMax; q += nt) {
      const unsigned long long v = q < take ? sk[q] : 0ull;
      list[q] = q < take ? make_uint2((uint32_t)(v >> 32), 0xFFFFFFFFu - (uint32_t)v) : make_uint2(0u, kListPad);
    }
    if (tid == 0) {
      *cnt_out = take;
      *bkey_out = T;
    }
    __syncthreads();
  } else {
    __syncthreads();  // the row's stores are visible to the whole CTA
    build_list_row<PREC, true>(P_row, n, list, cnt_out, bkey_out, scratch);
  }
}

// The collection threshold for a row's list from its previous bound bkey_prev:
// an entry's value changes by the evaporation keep^alpha (raised to AdaIR's
// exponent), so the previous T scaled by that and by 0.95 usually leaves a
// few hundred columns above it.  Any value gives the same list (see
// build_P_lists_row); 0xFFFFFFFF (none) when there is no previous bound.
__device__ __forceinline__ uint32_t list_guess(uint32_t bkey_prev, float keep, int alpha, float ig_now,
                                               float ig_prev) {
  if (bkey_prev == 0u || bkey_prev >= 0x7F800000u || !(keep > 0.0f) || !(ig_prev > 0.0f)) return 0xFFFFFFFFu;
  const float lx = log2f(__uint_as_float(bkey_prev)) / ig_prev + (float)alpha * log2f(keep);
  const float g = exp2f(ig_now * lx) * 0.95f;
  if (!(g > 0.0f) || !(g < 3.0e38f)) return 0xFFFFFFFFu;
  return __float_as_uint(g);
}

}  // namespace aco
