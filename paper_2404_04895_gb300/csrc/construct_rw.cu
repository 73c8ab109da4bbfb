// Roulette-wheel tour construction (Sec. 2.4: the classical selection that
// independent roulette replaces), in the exact integer reading the oracle
// states:
//   e    = floor(log2 of the largest unvisited p_j)
//   q_j  = floor(p_j * 2^(40 - e))
//   S    = sum of q_j over the unvisited j
//   u    = words 0 (high) and 1 (low) of Philox(counter (2^30, t, k, it))
//   v    = floor(u * S / 2^64)
//   next = the first unvisited j (column order) whose running sum exceeds v;
//          S = 0: the lowest unvisited j.
// Integer sums do not depend on their order, so the warp's parallel scan
// picks the same city as the oracle's sequential one.
//
// One warp per ant (n <= 16384).  Per step the row is staged in shared memory
// by cp.async; lane l owns the contiguous columns [l*B, (l+1)*B), B odd so
// that the lanes' reads fall in different banks; two passes over the block
// (maximum, then quanta), an exclusive warp scan of the lanes' 64-bit sums,
// and the lane whose range holds v walks its block in column order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "construct.cuh"
#include "internal.h"

namespace aco {

namespace {

constexpr int kRwMaxN = 16384;

__host__ __device__ inline int rw_block(int n) { return ((n + 31) / 32) | 1; }

__host__ __device__ inline size_t rw_smem_bytes(int n, int eb) {
  const size_t row = ((size_t)n * eb + 15) / 16 * 16;
  return row + (size_t)((n + 31) / 32) * 4;
}

// fp32 bit pattern of the stored element j of a staged row
template <int PREC>
__device__ __forceinline__ uint32_t rw_bits(const void* srow, int j) {
  if (PREC == ACO_FP32) return static_cast<const uint32_t*>(srow)[j];
  const uint32_t h = static_cast<const unsigned short*>(srow)[j];
  if (PREC == ACO_BF16) return h << 16;
  return __float_as_uint(__half2float(__ushort_as_half((unsigned short)h)));
}

// floor(log2 p) of a positive finite fp32 bit pattern
__device__ __forceinline__ int rw_exponent(uint32_t b) {
  const int eb = (int)(b >> 23);
  if (eb) return eb - 127;
  return (31 - __clz((int)(b & 0x7FFFFFu))) - 149;
}

// q = floor(p * 2^(40 - e)) for p <= 2^(e+1)
__device__ __forceinline__ uint64_t rw_quantum(uint32_t b, int e) {
  if (b == 0u) return 0ull;
  const int eb = (int)(b >> 23);
  const uint64_t mant = (uint64_t)(b & 0x7FFFFFu) | (eb ? 0x800000ull : 0ull);
  const int sh = (eb ? eb : 1) - 150 + 40 - e;
  if (sh >= 0) return mant << sh;
  return sh > -64 ? (mant >> -sh) : 0ull;
}

__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t x, int off) {
  const uint32_t lo = __shfl_up_sync(ACO_FULL_MASK, (uint32_t)x, off);
  const uint32_t hi = __shfl_up_sync(ACO_FULL_MASK, (uint32_t)(x >> 32), off);
  return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t x, int src) {
  const uint32_t lo = __shfl_sync(ACO_FULL_MASK, (uint32_t)x, src);
  const uint32_t hi = __shfl_sync(ACO_FULL_MASK, (uint32_t)(x >> 32), src);
  return ((uint64_t)hi << 32) | lo;
}

template <int PREC>
__global__ void __launch_bounds__(32) construct_rw_kernel(const void* __restrict__ Pv, int n, int ld, int m,
                                                          uint2 key, uint32_t it_arg,
                                                          const uint32_t* __restrict__ it_dev,
                                                          int32_t* __restrict__ tours, int32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint4 rsm[];
  const int k = blockIdx.x;
  if (k >= m) return;
  const int lane = threadIdx.x & 31;
  constexpr int EB = PREC == ACO_FP32 ? 4 : 2;
  const uint32_t it = it_dev ? *it_dev : it_arg;
  const int nchunks = (n * EB + 15) / 16;
  uint32_t* svis = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(rsm) + (size_t)nchunks * 16);
  const int nwords = (n + 31) / 32;
  const int B = rw_block(n);
  const int j0 = min(n, lane * B), j1 = min(n, j0 + B);
  int32_t* tour = tours + (size_t)k * n;
  const size_t row_bytes = (size_t)ld * EB;

  for (int q = lane; q < nwords; q += 32) svis[q] = 0u;
  __syncwarp();
  int cur = start_city(key, it, (uint32_t)k, n);
  if (lane == 0) {
    tour[0] = cur;
    svis[cur >> 5] |= 1u << (cur & 31);
  }
  __syncwarp();

  for (int t = 1; t < n; ++t) {
    const uint4* __restrict__ row4 = reinterpret_cast<const uint4*>(static_cast<const char*>(Pv) + (size_t)cur * row_bytes);
    for (int c = lane; c < nchunks; c += 32) cp_async16_pred(rsm + c, row4 + c, true);
    cp_async_wait_all();
    __syncwarp();  // every lane's copies have landed

    // pass 1: the largest unvisited value; each lane's first unvisited column
    uint32_t mx = 0u;
    int first = 0x7FFFFFFF;
    for (int j = j0; j < j1; ++j) {
      if ((svis[j >> 5] >> (j & 31)) & 1u) continue;
      first = min(first, j);
      mx = max(mx, rw_bits<PREC>(rsm, j));
    }
    mx = __reduce_max_sync(ACO_FULL_MASK, mx);
    const int lowest = (int)__reduce_min_sync(ACO_FULL_MASK, (uint32_t)first);
    int next = -1;
    if (mx == 0u) {
      next = lowest < n ? lowest : -1;  // every unvisited value is 0
    } else {
      const int e = rw_exponent(mx);
      // pass 2: this lane's sum of quanta, then an exclusive warp scan
      uint64_t s = 0ull;
      for (int j = j0; j < j1; ++j)
        if (!((svis[j >> 5] >> (j & 31)) & 1u)) s += rw_quantum(rw_bits<PREC>(rsm, j), e);
      uint64_t inc = s;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint64_t v = shfl_up_u64(inc, off);
        if (lane >= off) inc += v;
      }
      const uint64_t S = shfl_u64(inc, 31);
      const uint64_t excl = inc - s;
      const uint4 x = philox(make_uint4(1u << 30, (uint32_t)t, (uint32_t)k, it), key);
      const uint64_t u = ((uint64_t)x.x << 32) | (uint64_t)x.y;
      const uint64_t v = __umul64hi(u, S);
      const bool mine = excl <= v && v < inc;
      int pick = -1;
      if (mine) {
        uint64_t run = excl;
        for (int j = j0; j < j1; ++j) {
          if ((svis[j >> 5] >> (j & 31)) & 1u) continue;
          run += rw_quantum(rw_bits<PREC>(rsm, j), e);
          if (run > v) {
            pick = j;
            break;
          }
        }
      }
      const unsigned own = __ballot_sync(ACO_FULL_MASK, mine);
      next = own ? __shfl_sync(ACO_FULL_MASK, pick, __ffs(own) - 1) : -1;
    }
    if (next < 0 || next >= n) {  // cannot happen for valid input
      if (lane == 0 && err) atomicExch(err, kErrConstruct);
      break;
    }
    if (lane == 0) {
      tour[t] = next;
      svis[next >> 5] |= 1u << (next & 31);
    }
    __syncwarp();  // the bitmap update, and the staged row is free again
    cur = next;
  }
}

}  // namespace

int launch_construct_rw(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                        const uint32_t* it_dev, int32_t* tours, int32_t* err, cudaStream_t st) {
  if (n > kRwMaxN) return set_error(ACO_ERR_UNSUPPORTED, "roulette-wheel construction serves n <= %d", kRwMaxN);
  const int eb = prec == ACO_FP32 ? 4 : 2;
  const size_t smem = rw_smem_bytes(n, eb);
  switch (prec) {
    case ACO_FP32:
      construct_rw_kernel<ACO_FP32><<<m, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err);
      break;
    case ACO_BF16:
      construct_rw_kernel<ACO_BF16><<<m, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err);
      break;
    case ACO_FP16:
      construct_rw_kernel<ACO_FP16><<<m, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "construct_rw_kernel launch");
}

int prepare_construct_rw() {
  const int most = (int)rw_smem_bytes(kRwMaxN, 4);
  cudaError_t e = cudaFuncSetAttribute(construct_rw_kernel<ACO_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(construct_rw_kernel<ACO_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(construct_rw_kernel<ACO_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "cudaFuncSetAttribute(rw)");
}

}  // namespace aco
