// Per-row / per-ant / per-instance device functions of the iteration steps
// other than tour construction.  The single-instance kernels (kernels.cu) and
// the multi-instance kernels (batch.cu) are thin wrappers around them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

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

template <int PREC>
__device__ __forceinline__ void build_P_row(const float* __restrict__ tau_row,
                                            const float* __restrict__ H_row, int n, int ld, int i,
                                            int alpha, float inv_gamma, void* __restrict__ P_row,
                                            float* red /* [32] shared */) {
  const float4* t4 = reinterpret_cast<const float4*>(tau_row);
  const float4* h4 = reinterpret_cast<const float4*>(H_row);
  const int nq = ld >> 2;
  float scale = 1.0f;
  if (PREC == ACO_FP16) {
    float mx = 0.0f;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const float4 a = __ldg(t4 + q), b = __ldg(h4 + q);
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
    const float4 a = __ldg(t4 + q), b = __ldg(h4 + q);
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
// Eq. 3 + Eq. 2 for ant k (one warp): edge lengths D[p_t][p_{t+1}] gathered
// 32*U at a time, summed in fp64 in t order through shuffles (the order of a
// sequential loop); for city a = p_t the index mapping nbr[a][k] =
// (p_{t-1}, p_{t+1}); L_k and c_k = Q / L_k.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tour_length_ant(const double* __restrict__ D, int n,
                                                const int32_t* __restrict__ p, int m, int k,
                                                float Q, double* __restrict__ L,
                                                double* __restrict__ c,
                                                int32_t* __restrict__ nbr) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int base = 0; base < n; base += 32 * U) {
    double d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * 32 + lane;
      d[u] = 0.0;
      if (t < n) {
        const int a = p[t];
        const int b = p[t + 1 < n ? t + 1 : 0];
        const int pr = p[t > 0 ? t - 1 : n - 1];
        // tours come from the construction kernel; an entry out of range (only
        // after a failed construction, which the host reports) is skipped
        if ((unsigned)a < (unsigned)n && (unsigned)b < (unsigned)n) {
          d[u] = __ldg(D + (size_t)a * n + b);
          if (nbr) reinterpret_cast<int2*>(nbr)[(size_t)a * m + k] = make_int2(pr, b);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int cnt = min(32, n - (base + u * 32));
      for (int q = 0; q < cnt; ++q) s = __dadd_rn(s, __shfl_sync(ACO_FULL_MASK, d[u], q));
    }
  }
  if (lane == 0) {
    L[k] = s;
    if (c) c[k] = __ddiv_rn((double)Q, s);
  }
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
// Sec. 2.3 deterministic deposit of row a (one warp).  The row's increment
// Delta_a. is accumulated in fp64 shared memory; the row's 2m index-mapping
// entries (two neighbours per ant) are taken 16 ants at a time: lanes 0-15
// hold predecessors, lanes 16-31 successors.  __match_any_sync groups lanes
// with the same target column b; the lane of the lowest ant in a group adds
// the group's c_k to Delta_ab in ascending k, so every Delta_ab is summed in
// ascending ant order.  Columns in tiles of `tile`, ants in chunks of 1024.
// smem: tile doubles + kDepAntChunk * 16 bytes.
// ---------------------------------------------------------------------------
constexpr int kDepAntChunk = 1024;

__device__ __forceinline__ void deposit_row(float* __restrict__ row, int n,
                                            const int32_t* __restrict__ nbr_row,
                                            const double* __restrict__ c, int m, double keep,
                                            int tile, unsigned char* smem) {
  double* delta = reinterpret_cast<double*>(smem);            // [tile]
  double* cs = delta + tile;                                  // [kDepAntChunk]
  int2* items = reinterpret_cast<int2*>(cs + kDepAntChunk);   // [kDepAntChunk]
  const int lane = threadIdx.x & 31;
  for (int col0 = 0; col0 < n; col0 += tile) {
    const int cols = min(tile, n - col0);
    for (int q = lane; q < cols; q += 32) delta[q] = 0.0;
    for (int kb = 0; kb < m; kb += kDepAntChunk) {
      const int cnt = min(kDepAntChunk, m - kb);
      __syncwarp();
      const int2* src = reinterpret_cast<const int2*>(nbr_row) + kb;
#pragma unroll 4
      for (int q = lane; q < cnt; q += 32) {
        items[q] = __ldg(src + q);
        cs[q] = __ldg(c + kb + q);
      }
      __syncwarp();
      for (int k0 = 0; k0 < cnt; k0 += 16) {
        const int ai = lane & 15;  // ant k0 + ai
        const bool valid = k0 + ai < cnt;
        int b = -1;
        if (valid) {
          const int2 it = items[k0 + ai];
          b = (lane >> 4 ? it.y : it.x) - col0;
        }
        const bool in_tile = valid && b >= 0 && b < cols;
        const int key = in_tile ? b : -1 - lane;  // unique keys for idle lanes
        const unsigned grp = __match_any_sync(ACO_FULL_MASK, key);
        if (in_tile) {
          const unsigned ants = (grp & 0xFFFFu) | (grp >> 16);
          const int lead = __ffs(ants) - 1;
          if (lead == ai) {
            double sum = delta[b];
            unsigned rest = ants;
            while (rest) {
              const int i = __ffs(rest) - 1;
              rest &= rest - 1u;
              sum = __dadd_rn(sum, cs[k0 + i]);
            }
            delta[b] = sum;
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();
    // tau_ab <- fl32(fl64(keep * tau_ab) + Delta_ab), four columns per lane step
    const int nv = cols >> 2;
    float4* row4 = reinterpret_cast<float4*>(row + col0);
#pragma unroll 4
    for (int q = lane; q < nv; q += 32) {
      float4 v = row4[q];
      const double* dl = delta + 4 * q;
      v.x = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.x), dl[0]));
      v.y = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.y), dl[1]));
      v.z = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.z), dl[2]));
      v.w = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.w), dl[3]));
      row4[q] = v;
    }
    for (int q = 4 * nv + lane; q < cols; q += 32) {
      const int j = col0 + q;
      row[j] = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)row[j]), delta[q]));
    }
    __syncwarp();
  }
}

// fp64 shared bytes deposit_row needs for a tile of `tile` columns
__host__ __device__ inline size_t deposit_smem_bytes(int tile) {
  return (size_t)tile * 8 + (size_t)kDepAntChunk * 16;
}

// Column tile: the fp64 delta tile plus the per-chunk c and items fit 200 KB;
// a multiple of 4 so that every tile's columns start 16-byte aligned.
__host__ __device__ inline int deposit_tile(int n) {
  const int max_tile = ((200 * 1024 - kDepAntChunk * 16) / 8) & ~3;
  return n < max_tile ? n : max_tile;
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
// All threads of the CTA (blockDim.x <= 256); scratch: kListScratchWords
// shared words.
// ---------------------------------------------------------------------------
constexpr int kListTarget = 64;
constexpr int kListMax = 128;
constexpr int kListScratchWords = 256 + 8 + 2 * kListMax * 2;

template <int PREC>
__device__ __forceinline__ uint32_t p_key(const void* __restrict__ row, int j) {
  if (PREC == ACO_FP32) return __ldg(static_cast<const uint32_t*>(row) + j);
  const uint32_t h = __ldg(static_cast<const unsigned short*>(row) + j);
  if (PREC == ACO_BF16) return h << 16;
  return __float_as_uint(__half2float(__ushort_as_half((unsigned short)h)));
}

template <int PREC>
__device__ __forceinline__ void build_list_row(const void* __restrict__ P_row, int n,
                                               uint2* __restrict__ list, int* __restrict__ cnt_out,
                                               uint32_t* __restrict__ bkey_out,
                                               uint32_t* scratch) {
  uint32_t* hist = scratch;             // [256]
  uint32_t* sh = scratch + 256;         // [0] prefix, [1] need, [2] gt count, [3] eq count
  const int tid = threadIdx.x, nt = blockDim.x;
  if (n <= kListMax) {  // every column listed, bound 0; sorted below
    for (int j = tid; j < n; j += nt) list[j] = make_uint2(p_key<PREC>(P_row, j), (uint32_t)j);
    if (tid == 0) {
      *cnt_out = n;
      *bkey_out = 0u;
    }
    __syncthreads();
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(scratch + 256 + 8);
    for (int q = tid; q < kListMax; q += nt) {
      unsigned long long v = 0ull;
      if (q < n) {
        const uint2 e = list[q];
        v = ((unsigned long long)e.x << 32) | (unsigned long long)(0xFFFFFFFFu - e.y);
      }
      sk[q] = v;
    }
    __syncthreads();
    for (int size = 2; size <= kListMax; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int q = tid; q < kListMax; q += nt) {
          const int partner = q ^ stride;
          if (partner > q) {
            const bool desc = (q & size) == 0;
            const unsigned long long a = sk[q], b = sk[partner];
            if (desc ? (a < b) : (a > b)) {
              sk[q] = b;
              sk[partner] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int q = tid; q < n; q += nt) {
      const unsigned long long v = sk[q];
      list[q] = make_uint2((uint32_t)(v >> 32), 0xFFFFFFFFu - (uint32_t)v);
    }
    __syncthreads();
    return;
  }
  // 1. radix select of the kListTarget-th largest key T
  if (tid == 0) {
    sh[0] = 0u;
    sh[1] = kListTarget;
  }
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += nt) hist[b] = 0u;
    __syncthreads();
    const uint32_t prefix = sh[0];
    const uint32_t hi_mask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (int j = tid; j < n; j += nt) {
      const uint32_t key = p_key<PREC>(P_row, j);
      if ((key & hi_mask) == prefix) atomicAdd(&hist[(key >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t need = sh[1], cum = 0u;
      int digit = 0;
      for (int b = 255; b >= 0; --b) {
        if (cum + hist[b] >= need) {
          digit = b;
          break;
        }
        cum += hist[b];
      }
      sh[0] = prefix | ((uint32_t)digit << shift);
      sh[1] = need - cum;
    }
    __syncthreads();
  }
  const uint32_t T = sh[0];
  // 2. counts above and at T
  if (tid == 0) {
    sh[2] = 0u;
    sh[3] = 0u;
  }
  __syncthreads();
  uint32_t gt = 0, eq = 0;
  for (int j = tid; j < n; j += nt) {
    const uint32_t key = p_key<PREC>(P_row, j);
    gt += key > T;
    eq += key == T;
  }
  atomicAdd(&sh[2], gt);
  atomicAdd(&sh[3], eq);
  __syncthreads();
  const uint32_t n_gt = sh[2], n_eq = sh[3];
  const bool all_ties = n_gt + n_eq <= (uint32_t)kListMax;
  const uint32_t eq_take = all_ties ? n_eq : (uint32_t)kListMax - n_gt;
  // 3. compaction in column order: thread tid owns columns [tid*span, (tid+1)*span)
  const int span = (n + nt - 1) / nt;
  const int j0 = tid * span, j1 = min(n, j0 + span);
  uint32_t my_gt = 0, my_eq = 0;
  for (int j = j0; j < j1; ++j) {
    const uint32_t key = p_key<PREC>(P_row, j);
    my_gt += key > T;
    my_eq += key == T;
  }
  // exclusive scans over threads of the two counts (warp shuffles, then warp totals)
  const int lane = tid & 31, wid = tid >> 5;
  uint32_t inc_gt = my_gt, inc_eq = my_eq;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t vg = __shfl_up_sync(ACO_FULL_MASK, inc_gt, off);
    const uint32_t ve = __shfl_up_sync(ACO_FULL_MASK, inc_eq, off);
    if (lane >= off) {
      inc_gt += vg;
      inc_eq += ve;
    }
  }
  __syncthreads();
  if (lane == 31) {  // warp totals (hist is free again)
    hist[wid] = inc_gt;
    hist[32 + wid] = inc_eq;
  }
  __syncthreads();
  uint32_t before_gt = inc_gt - my_gt, before_eq = inc_eq - my_eq;
  for (int w = 0; w < wid; ++w) {
    before_gt += hist[w];
    before_eq += hist[32 + w];
  }
  // listed: all gt; eq in column order until eq_take
  uint32_t pos = before_gt + min(before_eq, eq_take);
  uint32_t eq_seen = before_eq;
  for (int j = j0; j < j1; ++j) {
    const uint32_t key = p_key<PREC>(P_row, j);
    if (key > T) {
      list[pos++] = make_uint2(key, (uint32_t)j);
    } else if (key == T) {
      if (eq_seen < eq_take) list[pos++] = make_uint2(key, (uint32_t)j);
      ++eq_seen;
    }
  }
  const int cnt = (int)(n_gt + eq_take);
  if (tid == 0) {
    *cnt_out = cnt;
    *bkey_out = all_ties ? T : T + 1u;
  }
  // 4. sort the list by key, descending (ties: lower column first): bitonic
  //    sort of kListMax 64-bit composite keys in shared memory
  __syncthreads();
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(scratch + 256 + 8);
  for (int q = tid; q < kListMax; q += nt) {
    unsigned long long v = 0ull;  // padding sorts last
    if (q < cnt) {
      const uint2 e = list[q];
      v = ((unsigned long long)e.x << 32) | (unsigned long long)(0xFFFFFFFFu - e.y);
    }
    sk[q] = v;
  }
  __syncthreads();
  for (int size = 2; size <= kListMax; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = tid; q < kListMax; q += nt) {
        const int partner = q ^ stride;
        if (partner > q) {
          const bool desc = (q & size) == 0;
          const unsigned long long a = sk[q], b = sk[partner];
          if (desc ? (a < b) : (a > b)) {
            sk[q] = b;
            sk[partner] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int q = tid; q < cnt; q += nt) {
    const unsigned long long v = sk[q];
    list[q] = make_uint2((uint32_t)(v >> 32), 0xFFFFFFFFu - (uint32_t)v);
  }
  __syncthreads();
}

}  // namespace aco
