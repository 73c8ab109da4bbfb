// Tour construction (Sec. 2.2 + 2.4): every ant walks n-1 independent-roulette
// steps over the shared transition matrix M_p.
//
// Layout of the work (one CTA = one ant, W warps, TPA = 32*W threads):
//   - Row P[cur] is cut into 16-byte chunks (V = 4 fp32 or 8 bf16/fp16
//     elements).  Thread g owns chunks c*TPA + g, c = 0..KC-1, for the whole
//     walk, and keeps the visited bits of its KC*V columns in registers.
//   - A step copies the thread's not-yet-fully-visited chunks of the row into
//     shared memory with 16-byte cp.async (coalesced: the warp moves 512
//     contiguous bytes per chunk index; every copy of the step is in flight
//     at once, whatever the register budget), waits for its own copies, then
//     reduces each 4-column group to its largest raw P.  Shared slot of chunk
//     c*TPA + g is its column-chunk index, so the row copy is dense.
//   - Exact pruning: a score is fl32(r * p) <= p because r < 1, so a column
//     whose p is below some candidate's exact score cannot win.  Each thread
//     first scores its largest group exactly (one Philox4x32-10 block covers
//     the group's 4 columns); the warp maximum of those scores is the
//     threshold, and only groups whose raw maximum reaches it are scored.
//     Skipping a counter-based draw changes no other draw, so the selected
//     city is exactly argmax over unvisited j of fl32(r_j * p_j), lowest j
//     on ties -- the same city a full scan selects.
//   - Warp shuffle argmax, then (W > 1) a shared-memory combine across warps.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "batch.cuh"
#include "common.cuh"
#include "lists.cuh"

namespace aco {

// 16-byte global -> shared copy (L2 only), issued only when `pred` holds.  A
// predicated instruction keeps all of a step's copies in one basic block.
__device__ __forceinline__ void cp_async16_pred(void* smem_dst, const void* gmem_src, bool pred) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
      "@p cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(dst),
      "l"(gmem_src), "r"((int)pred)
      : "memory");
}
// 16-byte read-only load into `v`, issued only when `pred` holds; otherwise v
// keeps its previous contents (no zeroing instructions).
__device__ __forceinline__ void ldg_pred_keep(uint4& v, const uint4* ptr, bool pred) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %5, 0;\n\t"
      "@p ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];\n\t}"
      : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
      : "l"(ptr), "r"((int)pred));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int PREC>
struct Elem;

template <>
struct Elem<ACO_FP32> {
  static constexpr int V = 4;      // elements per 16-byte chunk
  static constexpr int BYTES = 4;
  // fp32 bits of the largest element of group g (4 elements) of chunk d;
  // elements are >= 0, so unsigned order is numeric order.
  __device__ __forceinline__ static uint32_t group_max_bits(const uint4& d, int) {
    return max(__vimax3_u32(d.x, d.y, d.z), d.w);
  }
  __device__ __forceinline__ static float4 load_group(const char* row, int j0) {
    return __ldg(reinterpret_cast<const float4*>(row) + (j0 >> 2));
  }
  // the 4 values of group g of a 16-byte chunk
  __device__ __forceinline__ static float4 group_values(const uint4& d, int) {
    return make_float4(__uint_as_float(d.x), __uint_as_float(d.y), __uint_as_float(d.z),
                       __uint_as_float(d.w));
  }
};

__device__ __forceinline__ uint32_t vmax_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t swap_halves(uint32_t a) { return __byte_perm(a, 0, 0x1032); }

template <>
struct Elem<ACO_BF16> {
  static constexpr int V = 8;
  static constexpr int BYTES = 2;
  __device__ __forceinline__ static uint32_t group_max_bits(const uint4& d, int g) {
    const uint32_t m = g == 0 ? vmax_u16x2(d.x, d.y) : vmax_u16x2(d.z, d.w);
    return vmax_u16x2(m, swap_halves(m)) & 0xFFFF0000u;  // bf16 in the high half = fp32 bits
  }
  __device__ __forceinline__ static float4 group_values(const uint4& d, int g) {
    const uint32_t a = g == 0 ? d.x : d.z, b = g == 0 ? d.y : d.w;
    return make_float4(__uint_as_float(a << 16), __uint_as_float(a & 0xFFFF0000u),
                       __uint_as_float(b << 16), __uint_as_float(b & 0xFFFF0000u));
  }
  __device__ __forceinline__ static float4 load_group(const char* row, int j0) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(row) + (j0 >> 2));
    return group_values(make_uint4(v.x, v.y, 0u, 0u), 0);
  }
};

template <>
struct Elem<ACO_FP16> {
  static constexpr int V = 8;
  static constexpr int BYTES = 2;
  __device__ __forceinline__ static float h2f(uint32_t h) {
    return __half2float(__ushort_as_half((unsigned short)(h & 0xFFFFu)));
  }
  __device__ __forceinline__ static uint32_t group_max_bits(const uint4& d, int g) {
    const uint32_t m = g == 0 ? vmax_u16x2(d.x, d.y) : vmax_u16x2(d.z, d.w);
    return __float_as_uint(h2f(vmax_u16x2(m, swap_halves(m))));
  }
  __device__ __forceinline__ static float4 group_values(const uint4& d, int g) {
    const uint32_t a = g == 0 ? d.x : d.z, b = g == 0 ? d.y : d.w;
    return make_float4(h2f(a), h2f(a >> 16), h2f(b), h2f(b >> 16));
  }
  __device__ __forceinline__ static float4 load_group(const char* row, int j0) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(row) + (j0 >> 2));
    return group_values(make_uint4(v.x, v.y, 0u, 0u), 0);
  }
};

// Running argmax update with the lowest-index tie-break.
__device__ __forceinline__ void better(float s, int j, float& bs, int& bj) {
  if (s > bs || (s == bs && j < bj)) {
    bs = s;
    bj = j;
  }
}

// Order-preserving key of a candidate's score for unsigned warp reductions:
// 0 = no candidate, else fp32 bits + 1 (scores are >= 0).
__device__ __forceinline__ uint32_t score_key(float bs) {
  return bs >= 0.0f ? __float_as_uint(bs) + 1u : 0u;
}

// The first two rounds of row `row`'s candidate list and its bound, as loaded
// by one warp (rows are allocated and written whole: slots past the count
// hold (0, kListPad)).
struct ListRow {
  uint2 e, e_next;
  uint32_t lb;
  int row;
};

__device__ __forceinline__ ListRow load_list_row(const uint2* __restrict__ lists,
                                                 const uint32_t* __restrict__ lkey, int row) {
  const int lane = threadIdx.x & 31;
  const uint2* __restrict__ lrow = lists + (size_t)row * kListMax;
  ListRow L;
  L.e = __ldg(lrow + lane);
  L.e_next = __ldg(lrow + 32 + lane);
  L.lb = __ldg(lkey + row);
  L.row = row;
  return L;
}

// One step's candidate-list rounds (one warp; lists from build_list_row) on
// row L.row, whose first rounds L holds.  Entries are scored 32 at a time in
// value order, each round loaded one round ahead; an entry's visited bit is
// read while its Philox block is computed.  After a round, every entry not
// yet scored has a value <= the round's last one and every unlisted column a
// score key <= the row's bound, so the step is decided once the best score
// key exceeds both.  Returns the chosen column, or -1 when the list cannot
// decide; bs/bj then hold the best unvisited listed candidate (bs < 0: none),
// a threshold for the full scan.  (The full-scan kernel's list path; the lean
// kernel has its own rounds.)
__device__ __forceinline__ int list_rounds(const uint2* __restrict__ lists, const ListRow& L,
                                           const uint32_t* __restrict__ svis, const PhiloxKeys& key, uint32_t it,
                                           int k, int t, float& bs, int& bj) {
  const int lane = threadIdx.x & 31;
  const uint2* __restrict__ lrow = lists + (size_t)L.row * kListMax;
  uint2 e = L.e, e_next = L.e_next;
  // Rounds are written branch-free up to the decision so that the compiler
  // can interleave the Philox chain with the visited test; a padded slot
  // scores column 0 and is then ignored.
#pragma unroll 1
  for (int r = 0; r < kListMax / 32; ++r) {
    const bool valid = e.y != kListPad;
    const int j = valid ? (int)e.y : 0;
    const bool unvisited = valid && !((svis[j >> 5] >> (j & 31)) & 1u);
    const uint4 x = philox(make_uint4((uint32_t)(j >> 2), (uint32_t)t, (uint32_t)k, it), key);
    const unsigned vm = __ballot_sync(ACO_FULL_MASK, valid);
    // every entry after this round has a value <= this round's last one
    const bool more = (vm >> 31) != 0u && r + 1 < kListMax / 32;
    uint32_t rest = L.lb;
    if (more) rest = max(rest, __shfl_sync(ACO_FULL_MASK, e.x, 31) + 1u);
    const uint32_t w = (j & 2) ? ((j & 1) ? x.w : x.z) : ((j & 1) ? x.y : x.x);
    const float sc = __fmul_rn(uniform01(w), __uint_as_float(e.x));
    if (unvisited) better(sc, j, bs, bj);
    const uint32_t lk = __reduce_max_sync(ACO_FULL_MASK, score_key(bs));
    if (lk > rest)
      return (int)__reduce_min_sync(ACO_FULL_MASK, score_key(bs) == lk ? (uint32_t)bj : 0x7FFFFFFFu);
    if (!more) break;
    e = e_next;
    if (r + 2 < kListMax / 32) e_next = __ldg(lrow + 32 * (r + 2) + lane);
  }
  return -1;
}

// MODE_STAGED: a step's chunks go global -> shared memory by cp.async (all in
// flight regardless of registers; suits many chunks per thread).
// MODE_DIRECT: a step's chunks go straight into registers by predicated 16-byte
// loads (no shared-memory round trip; suits <= 12 chunks per thread, which
// the compiler keeps in flight together); the exact scorer re-reads its 16 or
// 8 bytes through L1.
constexpr int MODE_STAGED = 0;
constexpr int MODE_DIRECT = 1;

// The walk of ant k (all threads of the CTA call it together): start city, then
// n-1 steps over M_p (P, n x ld), tour written to tour[0..n-1].  red_s/red_j:
// [2][W] shared scratch; srow: [KC * 32 * W] shared chunks (MODE_STAGED only).
//
// Candidate lists (one warp per ant only; lists == nullptr disables them):
// each step first scores the unvisited entries of row cur's list (see
// build_list_row); when the best listed score key exceeds the row's bound the
// step is decided -- no unlisted column can reach or tie that score -- and the
// full scan is skipped; otherwise the full scan runs, seeded with the list's
// best candidate.  svis: n-bit shared visited bitmap the list phase reads.
template <int PREC, int W, int KC, int MODE>
__device__ __forceinline__ void construct_ant(const void* __restrict__ Pv, int n, int ld, uint2 key,
                                              uint32_t it, int k, int32_t* __restrict__ tour,
                                              int32_t* __restrict__ err, uint32_t (*red_s)[W],
                                              int (*red_j)[W], uint4* __restrict__ srow,
                                              const uint2* __restrict__ lists,
                                              const int* __restrict__ lcnt,
                                              const uint32_t* __restrict__ lkey,
                                              uint32_t* __restrict__ svis) {
  const bool use_list = W == 1 && lists != nullptr;
  using E = Elem<PREC>;
  constexpr int V = E::V;
  constexpr int G = V / 4;                // 4-column groups per chunk (one Philox block each)
  constexpr int NG = KC * G;              // groups per thread
  constexpr int MW = (KC * V + 31) / 32;  // visited-bit words per thread
  constexpr int TPA = 32 * W;             // threads per ant
  constexpr uint64_t GMASK = (1ull << G) - 1ull;
  constexpr int NA = NG < 4 ? NG : 4;     // independent accumulators for the top-2 keys
  static_assert(NG <= 64, "group masks are 64 bits");
  static_assert(NG <= 255, "group index packs into 8 bits");

  const int gl = threadIdx.x;
  const int lane = gl & 31;
  const int wi = gl >> 5;
  const char* __restrict__ P = static_cast<const char*>(Pv);
  const size_t row_bytes = (size_t)ld * E::BYTES;

  // visited bits: bit c*V + e  <->  column (c*TPA + gl)*V + e;
  // emptym bit gi: all 4 columns of group gi visited
  uint32_t vis[MW];
  uint64_t emptym = 0ull;
#pragma unroll
  for (int q = 0; q < MW; ++q) vis[q] = 0u;
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const int j0 = (c * TPA + gl) * V;
#pragma unroll
    for (int e = 0; e < V; ++e) {
      if (j0 + e >= n) vis[(c * V + e) >> 5] |= 1u << ((c * V + e) & 31);
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
      if (j0 + 4 * g >= n) emptym |= 1ull << (c * G + g);
  }
  auto mark = [&](int v) {
    const int cg = v / V;
    const int c = cg / TPA;
    const int bit = c * V + (v - cg * V);
    if (cg - c * TPA == gl) {
      uint32_t w = 0u;
#pragma unroll
      for (int q = 0; q < MW; ++q) {
        if (q == (bit >> 5)) {
          vis[q] |= 1u << (bit & 31);
          w = vis[q];
        }
      }
      if (((w >> (bit & 28)) & 0xFu) == 0xFu) emptym |= 1ull << (bit >> 2);
    }
  };
  auto nibble = [&](int bp) {  // visited bits of the 4-column group at bit bp
    uint32_t w = 0u;
#pragma unroll
    for (int q = 0; q < MW; ++q)
      if (q == (bp >> 5)) w = vis[q];
    return (w >> (bp & 31)) & 0xFu;
  };

  int cur = start_city(key, it, (uint32_t)k, n);
  const PhiloxKeys ks = philox_keys(key);
  if (gl == 0) tour[0] = cur;
  mark(cur);
  if (use_list) {
    for (int q = lane; q < (n + 31) / 32; q += 32) svis[q] = 0u;
    __syncwarp();
    if (lane == 0) svis[cur >> 5] |= 1u << (cur & 31);
    __syncwarp();
  }

  uint4 d[KC];  // MODE_DIRECT: the thread's chunks of the current row
#pragma unroll
  for (int c = 0; c < KC; ++c) d[c] = make_uint4(0u, 0u, 0u, 0u);

  for (int t = 1; t < n; ++t) {
    const char* __restrict__ row = P + (size_t)cur * row_bytes;
    const uint4* __restrict__ row4 = reinterpret_cast<const uint4*>(row);
    float bs = -1.0f;
    int bj = 0x7FFFFFFF;
    int next = -1;

    // 0. candidate list of row cur, sorted by value: rounds of 32 entries; after
    //    each round the next unscored entry (or the row's bound) bounds every
    //    column not scored yet
    if (use_list) {
      const ListRow L = load_list_row(lists, lkey, cur);
      next = list_rounds(lists, L, svis, ks, it, k, t, bs, bj);
    }

    if (next < 0) {  // full scan (seeded with the list's best candidate, if any)

    // 1. fetch every chunk with an unvisited column, 16 bytes each
    if (MODE == MODE_DIRECT) {
#pragma unroll
      for (int c = 0; c < KC; ++c)
        ldg_pred_keep(d[c], row4 + (c * TPA + gl), ((emptym >> (c * G)) & GMASK) != GMASK);
    } else {
#pragma unroll
      for (int c = 0; c < KC; ++c)
        cp_async16_pred(srow + c * TPA + gl, row4 + (c * TPA + gl),
                        ((emptym >> (c * G)) & GMASK) != GMASK);
      cp_async_wait_all();  // this thread's copies only: it reads nothing else
#pragma unroll
      for (int c = 0; c < KC; ++c) d[c] = srow[c * TPA + gl];
    }

    // 2. per group: raw maximum packed with the group index (-1: nothing unvisited);
    //    the thread's two largest keys, in NA independent accumulators
    int gkey[NG];
    int a1[NA], a2[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) a1[q] = a2[q] = -1;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int gi = c * G + g;
        const bool empty = (emptym >> gi) & 1ull;
        const uint32_t mb = E::group_max_bits(d[c], g);
        const int kk = empty ? -1 : (int)((mb & ~0xFFu) | (uint32_t)(0xFF - gi));
        gkey[gi] = kk;
        const int q = gi % NA;
        a2[q] = max(a2[q], min(a1[q], kk));
        a1[q] = max(a1[q], kk);
      }
    }
    int top = a1[0], second = a2[0];
#pragma unroll
    for (int q = 1; q < NA; ++q) {
      second = max(max(second, a2[q]), min(top, a1[q]));
      top = max(top, a1[q]);
    }

    auto score_group = [&](int gi) {
      const int c = gi / G, g = gi - c * G;
      const uint32_t nib = nibble(c * V + g * 4);
      if (nib == 0xFu) return;
      const int j0 = (c * TPA + gl) * V + g * 4;
      const float4 p = MODE == MODE_DIRECT ? E::load_group(row, j0)
                                           : E::group_values(srow[c * TPA + gl], g);
      const uint4 x = philox(make_uint4((uint32_t)(j0 >> 2), (uint32_t)t, (uint32_t)k, it), ks);
      if (!(nib & 1u)) better(__fmul_rn(uniform01(x.x), p.x), j0, bs, bj);
      if (!(nib & 2u)) better(__fmul_rn(uniform01(x.y), p.y), j0 + 1, bs, bj);
      if (!(nib & 4u)) better(__fmul_rn(uniform01(x.z), p.z), j0 + 2, bs, bj);
      if (!(nib & 8u)) better(__fmul_rn(uniform01(x.w), p.w), j0 + 3, bs, bj);
    };

    // 3. exact score of the top group; the warp's best exact score is the threshold
    const int top_gi = top >= 0 ? 0xFF - (top & 0xFF) : -1;
    if (top_gi >= 0) score_group(top_gi);
    const uint32_t thr_bits = __reduce_max_sync(ACO_FULL_MASK, bs >= 0.0f ? __float_as_uint(bs) : 0u);
    const int thr_key = (int)(thr_bits & ~0xFFu);

    // 4. other groups that can still reach the threshold (only if some thread's
    //    second-largest key reaches it)
    if (__any_sync(ACO_FULL_MASK, second >= thr_key)) {
      uint64_t surv = 0ull;
      if (second >= thr_key) {
#pragma unroll
        for (int gi = 0; gi < NG; ++gi)
          if (gkey[gi] >= thr_key && gi != top_gi) surv |= 1ull << gi;
      }
      while (__any_sync(ACO_FULL_MASK, surv != 0ull)) {
        if (surv) {
          const int gi = __ffsll((long long)surv) - 1;
          surv &= surv - 1ull;
          score_group(gi);
        }
      }
    }

    // 5. argmax across the warp (largest score, then lowest index), then across warps
    uint32_t wkey = __reduce_max_sync(ACO_FULL_MASK, score_key(bs));
    next = (int)__reduce_min_sync(ACO_FULL_MASK, score_key(bs) == wkey ? (uint32_t)bj : 0x7FFFFFFFu);
    if (W > 1) {
      if (lane == 0) {
        red_s[t & 1][wi] = wkey;
        red_j[t & 1][wi] = next;
      }
      __syncthreads();
      wkey = red_s[t & 1][0];
      next = red_j[t & 1][0];
#pragma unroll
      for (int w = 1; w < W; ++w) {
        const uint32_t ok = red_s[t & 1][w];
        const int oj = red_j[t & 1][w];
        if (ok > wkey || (ok == wkey && oj < next)) {
          wkey = ok;
          next = oj;
        }
      }
    }
    }  // full scan

    if (next < 0 || next >= n) {  // no unvisited city found: cannot happen for valid input
      if (gl == 0 && err) atomicExch(err, kErrConstruct);
      break;
    }
    if (gl == 0) tour[t] = next;
    mark(next);
    if (use_list) {
      if (lane == 0) svis[next >> 5] |= 1u << (next & 31);
      __syncwarp();
    }
    cur = next;
  }
}

// Dynamic shared memory: MODE_STAGED row chunks, then the list phase's bitmap.
template <int W, int KC, int MODE>
__host__ __device__ constexpr int srow_chunks() {
  return MODE == MODE_STAGED ? KC * 32 * W : 0;
}

template <int PREC, int W, int KC, int MODE>
__global__ void __launch_bounds__(32 * W) construct_kernel(
    const void* __restrict__ Pv, int n, int ld, int m, uint2 key, uint32_t it_arg,
    const uint32_t* __restrict__ it_dev, int32_t* __restrict__ tours, int32_t* __restrict__ err,
    const uint2* __restrict__ lists, const int* __restrict__ lcnt,
    const uint32_t* __restrict__ lkey) {
  __shared__ uint32_t red_s[2][W];
  __shared__ int red_j[2][W];
  extern __shared__ __align__(16) uint4 srow[];
  uint32_t* svis = reinterpret_cast<uint32_t*>(srow + srow_chunks<W, KC, MODE>());
  const int k = blockIdx.x;
  if (k >= m) return;
  const uint32_t it = it_dev ? *it_dev : it_arg;
  construct_ant<PREC, W, KC, MODE>(Pv, n, ld, key, it, k, tours + (size_t)k * n, err, red_s, red_j,
                                   srow, lists, lcnt, lkey, svis);
}

// Multi-instance construction: a persistent grid pulls work items (instance,
// ant) from a global counter; items are ordered by instance, instances by
// decreasing n, so the longest walks start first.  One launch covers every
// ant of every active instance of a batch.
// insts/ant_off point at the first instance of a size class of `count`
// instances; its items are ant_off[0] .. ant_off[0] + total - 1.
template <int PREC, int W, int KC, int MODE>
__global__ void __launch_bounds__(32 * W) batch_construct_kernel(
    const InstDev* __restrict__ insts, const int* __restrict__ ant_off, int count, int total,
    int* __restrict__ counter, int32_t* __restrict__ err) {
  const int base = __ldg(ant_off);
  __shared__ uint32_t red_s[2][W];
  __shared__ int red_j[2][W];
  __shared__ int item_s;
  extern __shared__ __align__(16) uint4 srow[];
  uint32_t* svis = reinterpret_cast<uint32_t*>(srow + srow_chunks<W, KC, MODE>());
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= total) break;
    const int i = find_instance(ant_off, count, base + item);
    const InstDev& I = insts[i];
    const int k = base + item - __ldg(ant_off + i);
    construct_ant<PREC, W, KC, MODE>(I.P, I.n, I.ld, I.key, *I.it, k, I.tours + (size_t)k * I.n, err,
                                     red_s, red_j, srow, I.lists, I.lcnt, I.lkey, svis);
  }
}

// Host launcher body for one precision: dispatch over the compiled shapes.
// The row buffer is KC * 32 * W * 16 bytes of dynamic shared memory.
#define ACO_CONSTRUCT_CASE(PREC, W, KC, MODE)                                              \
  if (warps == W && chunks == KC && mode == MODE) {                                         \
    const size_t smem_ = (size_t)srow_chunks<W, KC, MODE>() * 16 +                           \
                         (lists ? (size_t)((n + 127) / 128) * 16 : 0);                      \
    construct_kernel<PREC, W, KC, MODE><<<m, 32 * W, smem_, st>>>(                          \
        P, n, ld, m, key, it, it_dev, tours, err, W == 1 ? lists : nullptr, lcnt, lkey);     \
    const cudaError_t e_ = cudaGetLastError();                                              \
    return e_ == cudaSuccess ? ACO_OK : cuda_error(e_, "construct_kernel launch");          \
  }

}  // namespace aco

namespace aco {
#define ACO_BATCH_CONSTRUCT_CASE(PREC, W, KC, MODE)                                          \
  if (warps == W && chunks == KC && mode == MODE) {                                         \
    auto kern = batch_construct_kernel<PREC, W, KC, MODE>;                                  \
    const size_t smem_ = (size_t)srow_chunks<W, KC, MODE>() * 16 + (size_t)bitmap_bytes;    \
    static size_t occ_smem = (size_t)-1;                                                    \
    static int blocks_per_sm = 0;                                                           \
    if (occ_smem != smem_) {                                                                \
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_);  \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 32 * W, smem_);  \
      if (blocks_per_sm < 1) blocks_per_sm = 1;                                             \
      occ_smem = smem_;                                                                     \
    }                                                                                       \
    int grid_ = blocks_per_sm * num_sms;                                                    \
    if (grid_ > total) grid_ = total;                                                       \
    if (grid_ < 1) grid_ = 1;                                                               \
    kern<<<grid_, 32 * W, smem_, st>>>(insts, ant_off, count, total, counter, err);         \
    const cudaError_t e_ = cudaGetLastError();                                              \
    return e_ == cudaSuccess ? ACO_OK : cuda_error(e_, "batch_construct_kernel launch");    \
  }

// Opt every compiled shape in to its dynamic shared-memory size (once).
#define ACO_CONSTRUCT_PREPARE(PREC, W, KC, MODE)                                           \
  {                                                                                          \
    const cudaError_t e_ = cudaFuncSetAttribute(construct_kernel<PREC, W, KC, MODE>,         \
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                srow_chunks<W, KC, MODE>() * 16 + 8192);     \
    if (e_ != cudaSuccess) return cuda_error(e_, "cudaFuncSetAttribute(construct_kernel)");  \
  }
}  // namespace aco
