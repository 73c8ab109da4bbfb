// Lean tour construction: one warp per ant, candidate lists first, a compact
// full scan only when the list cannot decide a step (Sec. 2.2 + 2.4).
//
// State is the ant's visited bitmap in shared memory (n bits) and its current
// city; no per-lane visited registers, so the step stays short and light.
//   list step   the entries of row cur's sorted candidate list are scored in
//               rounds of 32 (one Philox4x32-10 block per entry); after each
//               round the round's last value -- and the row's bound -- bound
//               every column not yet scored, and the step is decided once the
//               best score key exceeds them (list_rounds, build_list_row)
//   full scan   (list undecided) the row is staged in shared memory by
//               cp.async; each lane walks its 4-column groups against a
//               threshold -- the warp's best listed score, raised by the lane's
//               own best score so far -- and scores exactly only the unvisited,
//               unlisted columns whose values reach it.
// Either way the chosen city is argmax over unvisited j of fl32(r_j * p_j),
// lowest j on ties, exactly as a plain scan of every candidate chooses.
#pragma once

#include "construct.cuh"

namespace aco {

// Dynamic shared memory of the lean kernel for n cities at element size eb:
// the staged row (chunks rounded to whole warps) and the visited bitmap.
__host__ __device__ inline size_t lean_smem_bytes(int n, int eb) {
  const int V = 16 / eb;
  const int chunks = (n + V - 1) / V;
  const int kc = (chunks + 31) / 32;
  return (size_t)kc * 32 * 16 + (size_t)((n + 127) / 128) * 16;
}

// Largest n the lean kernel serves (shared memory and 2 x 64-bit group masks).
__host__ __device__ inline int lean_max_n(int eb) { return eb == 4 ? 16384 : 16384; }

template <int PREC>
__device__ __forceinline__ void construct_ant_lean(const void* __restrict__ Pv, int n, int ld, uint2 key,
                                                   uint32_t it, int k, int32_t* __restrict__ tour,
                                                   int32_t* __restrict__ err,
                                                   const uint2* __restrict__ lists,
                                                   const int* __restrict__ lcnt,
                                                   const uint32_t* __restrict__ lkey,
                                                   uint4* __restrict__ srow, uint32_t* __restrict__ svis) {
  using E = Elem<PREC>;
  constexpr int V = E::V;
  constexpr int G = V / 4;
  const int lane = threadIdx.x & 31;
  const char* __restrict__ P = static_cast<const char*>(Pv);
  const size_t row_bytes = (size_t)ld * E::BYTES;
  const int nchunks = (n + V - 1) / V;
  const int kc = (nchunks + 31) / 32;  // chunks per lane
  const int nwords = (n + 31) / 32;

  // visited bits of the 4 columns of the group starting at j (columns >= n count as visited)
  auto group_nibble = [&](int j) -> uint32_t {
    uint32_t nib = (svis[j >> 5] >> (j & 31)) & 0xFu;
    if (j + 4 > n) nib |= (0xFu << max(0, n - j)) & 0xFu;
    return nib;
  };

  for (int q = lane; q < nwords; q += 32) svis[q] = 0u;
  __syncwarp();
  int cur = start_city(key, it, (uint32_t)k, n);
  const PhiloxKeys ks = philox_keys(key);
  if (lane == 0) svis[cur >> 5] |= 1u << (cur & 31);
  __syncwarp();
  // the tour is written 32 steps at a time: lane (t mod 32) keeps step t's city
  int tbuf = cur;

  ListRow lr, spec;
  lr.row = spec.row = -1;
  if (lists) lr = load_list_row(lists, lkey, cur);
  for (int t = 1; t < n; ++t) {
    const char* __restrict__ row = P + (size_t)cur * row_bytes;
    float bs = -1.0f;
    int bj = 0x7FFFFFFF;
    int next = -1;
    auto score4 = [&](int j0, float4 p, uint32_t nib) {
      const uint4 x = philox(make_uint4((uint32_t)(j0 >> 2), (uint32_t)t, (uint32_t)k, it), ks);
      if (!(nib & 1u)) better(__fmul_rn(uniform01(x.x), p.x), j0, bs, bj);
      if (!(nib & 2u)) better(__fmul_rn(uniform01(x.y), p.y), j0 + 1, bs, bj);
      if (!(nib & 4u)) better(__fmul_rn(uniform01(x.z), p.z), j0 + 2, bs, bj);
      if (!(nib & 8u)) better(__fmul_rn(uniform01(x.w), p.w), j0 + 3, bs, bj);
    };

    // ---- list step
    if (lists) next = list_rounds<true>(lists, lkey, lr, &spec, svis, ks, it, k, t, bs, bj);

    // ---- compact full scan
    if (next < 0) {
      const uint4* __restrict__ row4 = reinterpret_cast<const uint4*>(row);
      for (int c = 0; c < kc; ++c) {
        const int cg = c * 32 + lane;
        cp_async16_pred(srow + c * 32 + lane, row4 + cg, cg < nchunks);
      }
      cp_async_wait_all();  // this lane's copies only: it reads nothing else
      // Each lane walks its groups in column order against a threshold: the
      // warp's best listed score, raised by the lane's own best score so far.
      // A column whose value is below it cannot win or tie (a score never
      // exceeds its value), and a listed column -- value bits above the row's
      // bound - 1 -- was scored by the list rounds already, all of which ran.
      // Any other unvisited column is scored exactly at once.
      const uint32_t thr_warp = __reduce_max_sync(ACO_FULL_MASK, bs >= 0.0f ? __float_as_uint(bs) : 0u);
      const uint32_t hi = (lists && lr.lb) ? lr.lb - 1u : 0xFFFFFFFFu;
      const int nown = (nchunks - lane + 31) >> 5;  // chunks of this lane
#pragma unroll 4
      for (int c = 0; c < nown; ++c) {
        const uint4 v = srow[c * 32 + lane];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const uint32_t thr = max(thr_warp, bs >= 0.0f ? __float_as_uint(bs) : 0u);
          if (E::group_max_bits(v, g) < thr) continue;
          const int j0 = (c * 32 + lane) * V + 4 * g;
          if (j0 >= n) continue;
          const float4 p = E::group_values(v, g);
          auto out = [&](float x) -> uint32_t {
            const uint32_t b = __float_as_uint(x);
            return (b < thr || b > hi) ? 1u : 0u;
          };
          const uint32_t skip = group_nibble(j0) | out(p.x) | (out(p.y) << 1) | (out(p.z) << 2) | (out(p.w) << 3);
          if (skip != 0xFu) score4(j0, p, skip);
        }
      }
      const uint32_t wkey = __reduce_max_sync(ACO_FULL_MASK, score_key(bs));
      next = (int)__reduce_min_sync(ACO_FULL_MASK, score_key(bs) == wkey ? (uint32_t)bj : 0x7FFFFFFFu);
    }

    if (next < 0 || next >= n) {  // no unvisited city found: cannot happen for valid input
      if (lane == 0 && err) atomicExch(err, kErrConstruct);
      break;
    }
    if (lane == (t & 31)) tbuf = next;
    if ((t & 31) == 31 || t == n - 1) {
      const int tt = (t & ~31) + lane;
      if (tt <= t) tour[tt] = tbuf;
    }
    if (lane == 0) svis[next >> 5] |= 1u << (next & 31);
    __syncwarp();
    cur = next;
    // the next row's list: usually already in flight from the speculation
    if (lists && t + 1 < n) {
      if (spec.row == next)
        lr = spec;
      else
        lr = load_list_row(lists, lkey, next);
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(32) construct_lean_kernel(
    const void* __restrict__ Pv, int n, int ld, int m, uint2 key, uint32_t it_arg,
    const uint32_t* __restrict__ it_dev, int32_t* __restrict__ tours, int32_t* __restrict__ err,
    const uint2* __restrict__ lists, const int* __restrict__ lcnt, const uint32_t* __restrict__ lkey) {
  extern __shared__ __align__(16) uint4 lsm[];
  const int k = blockIdx.x;
  if (k >= m) return;
  const int eb = PREC == ACO_FP32 ? 4 : 2;
  const int chunks = (n + 16 / eb - 1) / (16 / eb);
  uint32_t* svis = reinterpret_cast<uint32_t*>(lsm + ((chunks + 31) / 32) * 32);
  const uint32_t it = it_dev ? *it_dev : it_arg;
  construct_ant_lean<PREC>(Pv, n, ld, key, it, k, tours + (size_t)k * n, err, lists, lcnt, lkey, lsm,
                           svis);
}

// Multi-instance form: persistent warps pull (instance, ant) items.
template <int PREC>
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
    const int k = base + item - __ldg(ant_off + i);
    construct_ant_lean<PREC>(I.P, I.n, I.ld, I.key, *I.it, k, I.tours + (size_t)k * I.n, err, I.lists,
                             I.lcnt, I.lkey, lsm, svis);
  }
}

}  // namespace aco
