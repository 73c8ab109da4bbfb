// Lean tour construction: candidate lists first, a compact full scan only
// when the list cannot decide a step (Sec. 2.2 + 2.4).  One warp walks one
// ant (kLeanAnts).
//
// State per ant is one visited flag byte per city in shared memory (marking a
// city is a single byte store, not a read-modify-write of a bitmap word), its
// current city and the first rounds of its current row's list.
//   list step   the entries of row cur's sorted candidate list are scored in
//               rounds of 32 (one Philox4x32-10 block per entry); after each
//               round the round's last value -- and the row's bound -- bound
//               every column not yet scored, and the step is decided once the
//               best score key exceeds them (build_list_row).  The first
//               round is one straight-line block (the argmax's two warp
//               reductions run whether or not the round decides), its Philox
//               rounds interleaved with the speculation below so that each
//               fills the other's waits; a later round whose entries are all
//               visited changes no score and costs no Philox block.
//   speculation in the first round the warp starts loading the lists of the
//               first two unvisited entries, one of which is usually next
//   full scan   (list undecided) the row is staged in shared memory by
//               cp.async; the warp walks it in blocks of 4 chunks per lane, a
//               branch-free test of every group against the lane's threshold
//               -- the warp's best listed score, raised by the lane's own best
//               score so far -- and scores exactly, only in blocks where some
//               lane has a group that reaches it, the unvisited, unlisted
//               columns whose values do.
// Either way the chosen city is argmax over unvisited j of fl32(r_j * p_j),
// lowest j on ties, exactly as a plain scan of every candidate chooses.
//
// One ant per warp: two ants per warp were measured 1.75x slower on GB300
// (n = 5000, m = 1024), and a second warp per ant that speculates while the
// first decides 1.45x slower -- the step is one latency-bound chain, and
// handing the speculated rows across warps through shared memory costs more
// than the speculation it moves.
#pragma once

#include "construct.cuh"

namespace aco {

// Visited flag of city j (one byte per city, at `flags`) and its marking.
__device__ __forceinline__ bool lean_visited(const uint32_t* flags, int j) {
  return reinterpret_cast<const volatile uint8_t*>(flags)[j] != 0;
}
__device__ __forceinline__ void lean_mark(uint32_t* flags, int j) { reinterpret_cast<volatile uint8_t*>(flags)[j] = 1; }

// Visited flags of one ant: one byte per city, rounded to 16 bytes (bytes past
// n stay 0; the scan masks columns >= n itself).
__host__ __device__ inline size_t lean_flag_bytes(int n) { return (size_t)((n + 15) / 16) * 16; }

// Dynamic shared memory of the lean kernel for n cities at element size eb
// and na ants per warp: the staged row (chunks rounded to whole warps) and one
// set of visited flags per ant.
__host__ __device__ inline size_t lean_smem_bytes(int n, int eb, int na = 1) {
  const int V = 16 / eb;
  const int chunks = (n + V - 1) / V;
  const int kc = (chunks + 31) / 32;
  return (size_t)kc * 32 * 16 + (size_t)na * lean_flag_bytes(n);
}

// Largest n the lean kernel serves (shared memory: 64 KB row + 16 KB flags).
__host__ __device__ inline int lean_max_n(int) { return 16384; }

// Ants per warp of the single-instance lean kernel.  Two ants per warp were
// measured 1.75x slower on GB300 (n = 5000, m = 1024): the warp-wide
// ballots, shuffles and reductions keep the two walks' chains from
// overlapping, and either ant's rare slow path stalls both.
constexpr int kLeanAnts = 1;

// The first round of row `row`'s list (lane l: entry l) and the row's bound:
// what every step needs.  Later rounds are loaded by lean_more_rounds, only
// for the few steps the first round does not decide.
struct ListHead {
  uint2 e;
  uint32_t lb;
  int row;
};

__device__ __forceinline__ ListHead load_list_head(const uint2* __restrict__ lists, const uint32_t* __restrict__ lkey,
                                                   int row) {
  ListHead L;
  L.e = __ldg(lists + (size_t)row * kListMax + (threadIdx.x & 31));
  L.lb = __ldg(lkey + row);
  L.row = row;
  return L;
}

// Rounds 1, 2, ... of a step's list after an undecided first round whose last
// entry was listed (so that more may follow); as list_rounds, with entries
// loaded two rounds ahead.
__device__ __forceinline__ int lean_more_rounds(const uint2* __restrict__ lists, const ListHead& L,
                                                 const uint32_t* __restrict__ svis, const PhiloxKeys& ks,
                                                 uint32_t it, int k, int t, float& bs, int& bj) {
  const int lane = threadIdx.x & 31;
  constexpr int R = kListMax / 32;
  const uint2* __restrict__ lrow = lists + (size_t)L.row * kListMax;
  uint2 e = __ldg(lrow + 32 + lane);
  uint2 e2 = R > 2 ? __ldg(lrow + 64 + lane) : e;
  uint2 e3 = R > 3 ? __ldg(lrow + 96 + lane) : e;
  uint32_t lk = __reduce_max_sync(ACO_FULL_MASK, score_key(bs));
#pragma unroll 1
  for (int r = 1; r < R; ++r) {
    const bool valid = e.y != kListPad;
    const unsigned vm = __ballot_sync(ACO_FULL_MASK, valid);
    if (vm == 0u) break;  // past the last entry
    const int j = valid ? (int)e.y : 0;
    const bool unvisited = valid && !lean_visited(svis, j);
    const unsigned un = __ballot_sync(ACO_FULL_MASK, unvisited);
    const bool more = (vm >> 31) != 0u && r + 1 < R;
    uint32_t rest = L.lb;
    if (more) rest = max(rest, __shfl_sync(ACO_FULL_MASK, e.x, 31) + 1u);
    if (un) {  // a round whose entries are all visited changes no score
      const uint4 x = philox(make_uint4((uint32_t)(j >> 2), (uint32_t)t, (uint32_t)k, it), ks);
      const uint32_t w = (j & 2) ? ((j & 1) ? x.w : x.z) : ((j & 1) ? x.y : x.x);
      const float sc = __fmul_rn(uniform01(w), __uint_as_float(e.x));
      if (unvisited) better(sc, j, bs, bj);
      lk = __reduce_max_sync(ACO_FULL_MASK, score_key(bs));
    }
    if (lk > rest)
      return (int)__reduce_min_sync(ACO_FULL_MASK, score_key(bs) == lk ? (uint32_t)bj : 0x7FFFFFFFu);
    if (!more) break;
    e = e2;
    e2 = e3;
    if (r + 3 < R) e3 = __ldg(lrow + 32 * (r + 3) + lane);
  }
  return -1;
}

// The compact full scan of row `row` for one ant (one warp): every unvisited,
// unlisted column whose value reaches the threshold is scored exactly; bs/bj
// enter with the best listed candidate.  hi: largest value bits a column may
// have and still be unlisted.  Returns the argmax (lowest column on ties).
template <int PREC>
__device__ __forceinline__ int lean_full_scan(const char* __restrict__ row, int n, uint32_t hi,
                                              const uint32_t* __restrict__ svis, uint4* __restrict__ srow,
                                              const PhiloxKeys& ks, uint32_t it, int k, int t, float& bs,
                                              int& bj) {
  using E = Elem<PREC>;
  constexpr int V = E::V;
  constexpr int G = V / 4;
  const int lane = threadIdx.x & 31;
  const int nchunks = (n + V - 1) / V;
  const int kc = (nchunks + 31) / 32;
  // visited flags of the 4 columns of the group starting at j (a multiple of
  // 4) as bits 0..3; columns >= n count as visited
  auto group_nibble = [&](int j) -> uint32_t {
    const uint32_t wv = *reinterpret_cast<const volatile uint32_t*>(reinterpret_cast<const uint8_t*>(svis) + j);
    uint32_t nib = (((wv & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
    if (j + 4 > n) nib |= (0xFu << max(0, n - j)) & 0xFu;
    return nib;
  };
  auto score4 = [&](int j0, float4 p, uint32_t skip) {
    const uint4 x = philox(make_uint4((uint32_t)(j0 >> 2), (uint32_t)t, (uint32_t)k, it), ks);
    if (!(skip & 1u)) better(__fmul_rn(uniform01(x.x), p.x), j0, bs, bj);
    if (!(skip & 2u)) better(__fmul_rn(uniform01(x.y), p.y), j0 + 1, bs, bj);
    if (!(skip & 4u)) better(__fmul_rn(uniform01(x.z), p.z), j0 + 2, bs, bj);
    if (!(skip & 8u)) better(__fmul_rn(uniform01(x.w), p.w), j0 + 3, bs, bj);
  };
  const uint4* __restrict__ row4 = reinterpret_cast<const uint4*>(row);
  for (int c = 0; c < kc; ++c) {
    const int cg = c * 32 + lane;
    cp_async16_pred(srow + c * 32 + lane, row4 + cg, cg < nchunks);
  }
  cp_async_wait_all();  // this lane's copies only: it reads nothing else
  // Each lane walks its groups in column order against a threshold: the
  // warp's best listed score, raised by the lane's own best score so far.
  // A column whose value is below it cannot win or tie (a score never
  // exceeds its value), and a listed column -- value bits above hi -- was
  // scored by the list rounds already, all of which ran.
  uint32_t thr_warp = __reduce_max_sync(ACO_FULL_MASK, bs >= 0.0f ? __float_as_uint(bs) : 0u);
  const int nown = (nchunks - lane + 31) >> 5;  // chunks of this lane
  // blocks of 4 chunks: a branch-free test of every group; the per-column
  // work runs only in blocks where some lane has a group that reaches its
  // threshold (a warp-uniform branch)
  for (int c0 = 0; c0 < kc; c0 += 4) {
    uint4 v[4];
    uint32_t hit = 0u;
    const uint32_t thr0 = max(thr_warp, bs >= 0.0f ? __float_as_uint(bs) : 0u);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      v[u] = c < nown ? srow[c * 32 + lane] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int g = 0; g < G; ++g)
        hit |= (c < nown && E::group_max_bits(v[u], g) >= thr0) ? (1u << (u * G + g)) : 0u;
    }
    if (__any_sync(ACO_FULL_MASK, hit != 0u)) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (!((hit >> (u * G + g)) & 1u)) continue;
          const uint32_t thr = max(thr_warp, bs >= 0.0f ? __float_as_uint(bs) : 0u);
          if (E::group_max_bits(v[u], g) < thr) continue;
          const int j0 = ((c0 + u) * 32 + lane) * V + 4 * g;
          if (j0 >= n) continue;
          const float4 p = E::group_values(v[u], g);
          auto out = [&](float x) -> uint32_t {
            const uint32_t b = __float_as_uint(x);
            return (b < thr || b > hi) ? 1u : 0u;
          };
          const uint32_t skip = group_nibble(j0) | out(p.x) | (out(p.y) << 1) | (out(p.z) << 2) | (out(p.w) << 3);
          if (skip != 0xFu) score4(j0, p, skip);
        }
      }
    }
  }
  const uint32_t wkey = __reduce_max_sync(ACO_FULL_MASK, score_key(bs));
  const int next = (int)__reduce_min_sync(ACO_FULL_MASK, score_key(bs) == wkey ? (uint32_t)bj : 0x7FFFFFFFu);
  __syncwarp();  // the staged row is free again
  return next;
}

// Step probes (PROBE instantiations only): the SM clock (%clock) read after
// `dep` is available, so that the stamp cannot come before the value.
__device__ __forceinline__ uint32_t clock_after(uint32_t dep) {
  uint32_t t;
  asm volatile("mov.u32 %0, %%clock;" : "=r"(t) : "r"(dep) : "memory");
  return t;
}

// Probe record of one step of one ant: 8 words.
//   [0] clock at the step's start   [1..6] cycles from it until: the step's
//   first list entry is available, its Philox block is done, the speculative
//   list loads are issued, the first round's decision, the slow paths'
//   decision, the end of the step's bookkeeping   [7] flags: 1 the first
//   round decided, 2 later list rounds ran, 4 a full scan ran, 8/16 the next
//   list came from speculation slot 0/1 (else it was loaded after the step).
constexpr int kProbeWords = 8;

// NA ants walked by one warp: ants k[q], tours tour[q], visited flags svis[q].
// FULL0: every list has >= 32 entries (n >= 32: a list holds at least
// min(kListTarget, n) of the row's n columns), so its first round has no
// padded slot.  LISTS: candidate lists are given (else every step is a
// compact full scan).  Both are compile-time: with them fixed the step's
// control flow is straight (measured 17-19% faster than testing them per step).
// PROBE: lane 0 of ant 0 writes one probe record per step to probe[t * 8]
// (NA == 1; a measurement build: the clock reads change the schedule a little).
template <int PREC, int NA, bool FULL0, bool LISTS, bool PROBE = false>
__device__ __forceinline__ void construct_ants_lean(const void* __restrict__ Pv, int n, int ld, uint2 key,
                                                    uint32_t it, const int* k, int32_t* const* tour,
                                                    int32_t* __restrict__ err,
                                                    const uint2* __restrict__ lists,
                                                    const uint32_t* __restrict__ lkey,
                                                    uint4* __restrict__ srow, uint32_t* const* svis,
                                                    uint32_t* __restrict__ probe = nullptr) {
  using E = Elem<PREC>;
  const int lane = threadIdx.x & 31;
  const char* __restrict__ P = static_cast<const char*>(Pv);
  const size_t row_bytes = (size_t)ld * E::BYTES;
  const PhiloxKeys ks = philox_keys(key);

  int cur[NA];
  ListHead lr[NA], sp[NA][2];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    for (int w = lane; w < (int)(lean_flag_bytes(n) / 4); w += 32) svis[q][w] = 0u;
    cur[q] = start_city(key, it, (uint32_t)k[q], n);
    lr[q].row = sp[q][0].row = sp[q][1].row = -1;
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    if (lane == 0) {
      lean_mark(svis[q], cur[q]);
      tour[q][0] = cur[q];
    }
    if (LISTS) lr[q] = load_list_head(lists, lkey, cur[q]);
  }
  __syncwarp();

  for (int t = 1; t < n; ++t) {
    int next[NA];
    float bs[NA];
    int bj[NA];
    bool more[NA];
    uint32_t pr[kProbeWords] = {};
    if constexpr (PROBE) pr[0] = clock_after(0u);
    // ---- first list round of every ant: one straight-line block
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      bs[q] = -1.0f;
      bj[q] = 0x7FFFFFFF;
      next[q] = -1;
      more[q] = false;
      if (LISTS) {
        const uint2 e = lr[q].e;
        if constexpr (PROBE) pr[1] = clock_after(e.y) - pr[0];
        const bool valid = FULL0 || e.y != kListPad;
        const int j = FULL0 ? (int)e.y : (valid ? (int)e.y : 0);
        uint4 xc = make_uint4((uint32_t)(j >> 2), (uint32_t)t, (uint32_t)k[q], it);
        const bool unvisited = valid && !lean_visited(svis[q], j);
        philox_round(xc, ks, 0);
        philox_round(xc, ks, 1);
        philox_round(xc, ks, 2);
        const unsigned vm = FULL0 ? 0xFFFFFFFFu : __ballot_sync(ACO_FULL_MASK, valid);
        const unsigned un = __ballot_sync(ACO_FULL_MASK, unvisited);
        philox_round(xc, ks, 3);
        philox_round(xc, ks, 4);
        const unsigned un2 = un & (un - 1u);
        const int sj = __shfl_sync(ACO_FULL_MASK, j, __ffs(un) - 1);
        philox_round(xc, ks, 5);
        philox_round(xc, ks, 6);
        const int sj2 = __shfl_sync(ACO_FULL_MASK, j, __ffs(un2) - 1);
        philox_round(xc, ks, 7);
        sp[q][0] = load_list_head(lists, lkey, sj);
        sp[q][1] = load_list_head(lists, lkey, sj2);
        if constexpr (PROBE) pr[3] = clock_after((uint32_t)sj2) - pr[0];
        if (!un) sp[q][0].row = -1;
        if (!un2) sp[q][1].row = -1;
        more[q] = (vm >> 31) != 0u && kListMax / 32 > 1;
        uint32_t rest = lr[q].lb;
        if (more[q]) rest = max(rest, __shfl_sync(ACO_FULL_MASK, e.x, 31) + 1u);
        philox_round(xc, ks, 8);
        philox_round(xc, ks, 9);
        const uint4 x = xc;
        if constexpr (PROBE) pr[2] = clock_after(x.x ^ x.y ^ x.z ^ x.w) - pr[0];
        const uint32_t w = (j & 2) ? ((j & 1) ? x.w : x.z) : ((j & 1) ? x.y : x.x);
        const float sc = __fmul_rn(uniform01(w), __uint_as_float(e.x));
        {
          // better(sc, j) against the round's start (-1, none), written out:
          // every unvisited finite score is taken, a NaN never
          const bool take = unvisited && sc > -1.0f;
          bs[q] = take ? sc : -1.0f;
          bj[q] = take ? j : 0x7FFFFFFF;
        }
        const uint32_t lk = __reduce_max_sync(ACO_FULL_MASK, score_key(bs[q]));
        const int win = (int)__reduce_min_sync(ACO_FULL_MASK, score_key(bs[q]) == lk ? (uint32_t)bj[q] : 0x7FFFFFFFu);
        if (lk > rest) next[q] = win;
        if constexpr (PROBE) {
          pr[4] = clock_after((uint32_t)win) - pr[0];
          pr[7] |= next[q] >= 0 ? 1u : 0u;
        }
      }
    }
    // ---- later rounds and full scans, ant by ant (rare)
#pragma unroll
    for (int q = 0; q < NA; ++q) {

      if (next[q] < 0 && LISTS && (FULL0 || more[q])) {
        next[q] = lean_more_rounds(lists, lr[q], svis[q], ks, it, k[q], t, bs[q], bj[q]);
        if constexpr (PROBE) pr[7] |= 2u;
      }
      if (next[q] < 0) {
        const uint32_t hi = (LISTS && lr[q].lb) ? lr[q].lb - 1u : 0xFFFFFFFFu;
        next[q] = lean_full_scan<PREC>(P + (size_t)cur[q] * row_bytes, n, hi, svis[q], srow, ks, it, k[q], t,
                                       bs[q], bj[q]);
        if constexpr (PROBE) pr[7] |= 4u;
      }
    }
    if constexpr (PROBE) pr[5] = clock_after((uint32_t)next[0]) - pr[0];
    // ---- bookkeeping
    bool bad = false;
#pragma unroll
    for (int q = 0; q < NA; ++q) bad = bad || next[q] < 0 || next[q] >= n;
    if (bad) {  // no unvisited city found: cannot happen for valid input
      if (lane == 0 && err) atomicExch(err, kErrConstruct);
      break;
    }
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      if (lane == 0) tour[q][t] = next[q];
      lean_mark(svis[q], next[q]);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      cur[q] = next[q];
      // the next row's list: usually already in flight from the speculation
      if (LISTS) {  // after the last step: one unused load of a valid row
        if (sp[q][0].row == next[q]) {
          lr[q] = sp[q][0];
          if constexpr (PROBE) pr[7] |= 8u;
        } else if (sp[q][1].row == next[q]) {
          lr[q] = sp[q][1];
          if constexpr (PROBE) pr[7] |= 16u;
        } else {
          lr[q] = load_list_head(lists, lkey, next[q]);
        }
      }
    }
    if constexpr (PROBE) {
      pr[6] = clock_after((uint32_t)cur[0]) - pr[0];
      if (lane == 0) {
        uint4* o = reinterpret_cast<uint4*>(probe + (size_t)t * kProbeWords);
        o[0] = make_uint4(pr[0], pr[1], pr[2], pr[3]);
        o[1] = make_uint4(pr[4], pr[5], pr[6], pr[7]);
      }
    }
  }
}

// One warp per kLeanAnts ants (the last warp of an odd m walks its ant twice
// and writes the same tour twice).  FULL0, LISTS as construct_ants_lean.
template <int PREC, bool FULL0, bool LISTS>
__global__ void __launch_bounds__(32) construct_lean_kernel(
    const void* __restrict__ Pv, int n, int ld, int m, uint2 key, uint32_t it_arg,
    const uint32_t* __restrict__ it_dev, int32_t* __restrict__ tours, int32_t* __restrict__ err,
    const uint2* __restrict__ lists, const int* __restrict__ lcnt, const uint32_t* __restrict__ lkey) {
  extern __shared__ __align__(16) uint4 lsm[];
  (void)lcnt;
  const int k0 = blockIdx.x * kLeanAnts;
  if (k0 >= m) return;
  const int eb = PREC == ACO_FP32 ? 4 : 2;
  const int chunks = (n + 16 / eb - 1) / (16 / eb);
  char* bitmaps = reinterpret_cast<char*>(lsm + ((chunks + 31) / 32) * 32);
  int k[kLeanAnts];
  int32_t* tour[kLeanAnts];
  uint32_t* svis[kLeanAnts];
#pragma unroll
  for (int q = 0; q < kLeanAnts; ++q) {
    k[q] = min(k0 + q, m - 1);
    tour[q] = tours + (size_t)k[q] * n;
    svis[q] = reinterpret_cast<uint32_t*>(bitmaps + q * lean_flag_bytes(n));
  }
  const uint32_t it = it_dev ? *it_dev : it_arg;
  construct_ants_lean<PREC, kLeanAnts, FULL0, LISTS>(Pv, n, ld, key, it, k, tour, err, lists, lkey, lsm, svis);
}

// The lean kernel with step probes: every ant walks as in construct_lean_kernel
// (lists, n >= 32); ant `probe_ant` also writes one probe record per step to
// probe[t * kProbeWords] (t = 1 .. n-1).
template <int PREC>
__global__ void __launch_bounds__(32) construct_lean_probe_kernel(
    const void* __restrict__ Pv, int n, int ld, int m, uint2 key, uint32_t it, int32_t* __restrict__ tours,
    int32_t* __restrict__ err, const uint2* __restrict__ lists, const uint32_t* __restrict__ lkey, int probe_ant,
    uint32_t* __restrict__ probe) {
  extern __shared__ __align__(16) uint4 lsm[];
  const int k0 = blockIdx.x;
  if (k0 >= m) return;
  const int eb = PREC == ACO_FP32 ? 4 : 2;
  const int chunks = (n + 16 / eb - 1) / (16 / eb);
  uint32_t* svis[1] = {reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(lsm + ((chunks + 31) / 32) * 32))};
  int k[1] = {k0};
  int32_t* tour[1] = {tours + (size_t)k0 * n};
  if (k0 == probe_ant)
    construct_ants_lean<PREC, 1, true, true, true>(Pv, n, ld, key, it, k, tour, err, lists, lkey, lsm, svis, probe);
  else
    construct_ants_lean<PREC, 1, true, true, false>(Pv, n, ld, key, it, k, tour, err, lists, lkey, lsm, svis);
}

// Multi-instance form: persistent warps pull (instance, ant) items; every
// instance has candidate lists.  FULL0: every instance has n >= 32.
template <int PREC, bool FULL0>
__global__ void __launch_bounds__(32) batch_construct_lean_kernel(
    const InstDev* __restrict__ insts, const int* __restrict__ ant_off, int count, int total,
    int* __restrict__ counter, int32_t* __restrict__ err, int max_n) {
  extern __shared__ __align__(16) uint4 lsm[];
  const int eb = PREC == ACO_FP32 ? 4 : 2;
  const int max_chunks = (max_n + 16 / eb - 1) / (16 / eb);
  uint32_t* svis = reinterpret_cast<uint32_t*>(lsm + ((max_chunks + 31) / 32) * 32);
  const int base = __ldg(ant_off);
  for (;;) {
    int item = 0;
    if ((threadIdx.x & 31) == 0) item = atomicAdd(counter, 1);
    item = __shfl_sync(ACO_FULL_MASK, item, 0);
    if (item >= total) break;
    const int i = find_instance(ant_off, count, base + item);
    const InstDev& I = insts[i];
    int k[1] = {base + item - __ldg(ant_off + i)};
    int32_t* tour[1] = {I.tours + (size_t)k[0] * I.n};
    uint32_t* sv[1] = {svis};
    construct_ants_lean<PREC, 1, FULL0, true>(I.P, I.n, I.ld, I.key, *I.it, k, tour, err, I.lists, I.lkey, lsm, sv);
  }
}

}  // namespace aco
