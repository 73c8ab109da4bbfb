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
// One CTA of kRwThreads threads per ant (n <= 16384).  Per step the row is
// staged in shared memory by one TMA bulk copy (cp.async.bulk, completion on
// an mbarrier); thread q owns the contiguous columns [q*B, (q+1)*B), B a
// multiple of 4 with B/4 odd, read 4 columns at a time (one vector load of
// values, one word of flags) so that the threads of a load phase hit
// different banks; two passes over the block (maximum, then quanta), a
// block-wide exclusive scan of the threads' 64-bit sums, and the thread whose
// range holds v walks its block in column order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "batch.cuh"
#include "common.cuh"
#include "construct.cuh"
#include "internal.h"

namespace aco {

namespace {

constexpr int kRwThreads = 256;
constexpr uint32_t kRwSpin = kRwWaitPolls;  // bound on the wait that drains a copy after a give-up

__host__ __device__ inline int rw_block(int n) {
  const int q = (n + kRwThreads - 1) / kRwThreads;  // columns per thread, at least
  return 4 * (((q + 3) / 4) | 1);
}
__host__ __device__ inline size_t rw_row_bytes(int n, int eb) { return ((size_t)n * eb + 15) / 16 * 16; }
__host__ __device__ inline size_t rw_flag_bytes(int n) { return ((size_t)n + 15) / 16 * 16; }
// control block after the row and the flags: the mbarrier (8 bytes, 16
// reserved), the warps' 64-bit sums, maxima and lowest unvisited columns, the
// chosen column
constexpr int kRwCtlBytes = 16 + 8 * (kRwThreads / 32) + 4 * (kRwThreads / 32) + 4 * (kRwThreads / 32) + 4;
static_assert(kRwCtlBytes <= 256, "control block");
// staged row, visited flags (one byte per city), control block
__host__ __device__ inline size_t rw_smem_bytes(int n, int eb) { return rw_row_bytes(n, eb) + rw_flag_bytes(n) + 256; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on the mbarrier.  The proxy fence
// orders this thread's (and, after a CTA barrier, every thread's) earlier
// generic accesses to the buffer before the copy's writes.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Waits until the mbarrier's phase `parity` has completed, for at most
// `polls` polls; false if it has not.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t polls) {
  for (uint32_t i = 0; i < polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// fp32 bit patterns of the stored elements j..j+3 of a staged row (j a
// multiple of 4: a 16- or 8-byte aligned load)
template <int PREC>
__device__ __forceinline__ void rw_bits4(const void* srow, int j, uint32_t b[4]) {
  if (PREC == ACO_FP32) {
    const uint4 v = *reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(srow) + j);
    b[0] = v.x;
    b[1] = v.y;
    b[2] = v.z;
    b[3] = v.w;
  } else {
    const uint2 v = *reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(srow) + j);
    const uint32_t h[4] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      b[i] = PREC == ACO_BF16 ? h[i] << 16 : __float_as_uint(__half2float(__ushort_as_half((unsigned short)h[i])));
  }
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

// The tour of ant k (one CTA of kRwThreads threads; `rsm` holds
// rw_smem_bytes(n) bytes of dynamic shared memory).  Each step waits at most
// `polls` polls for its row copy; when that runs out the CTA sets *err to
// kErrTimeout, drains the copy (a wait of kRwSpin polls) and stops.
template <int PREC>
__device__ __forceinline__ void rw_ant(const void* __restrict__ Pv, int n, int ld, uint2 key, uint32_t it, int k,
                                       int32_t* __restrict__ tour, int32_t* __restrict__ err, uint32_t polls,
                                       uint4* rsm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kRwThreads / 32;
  constexpr int EB = PREC == ACO_FP32 ? 4 : 2;
  char* sbase = reinterpret_cast<char*>(rsm);
  const uint32_t row_bytes = (uint32_t)rw_row_bytes(n, EB);  // <= ld * EB: a row's padded span
  volatile uint8_t* flags = reinterpret_cast<uint8_t*>(sbase + row_bytes);
  char* ctl = sbase + row_bytes + rw_flag_bytes(n);
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctl);
  unsigned long long* wsum = reinterpret_cast<unsigned long long*>(ctl + 16);  // [NW]
  uint32_t* wmax = reinterpret_cast<uint32_t*>(ctl + 16 + 8 * NW);              // [NW]
  int* wfirst = reinterpret_cast<int*>(ctl + 16 + 12 * NW);                     // [NW]
  volatile int* spick = reinterpret_cast<int*>(ctl + 16 + 16 * NW);
  const uint32_t sbar = smem_addr(bar), srow = smem_addr(sbase);
  const int B = rw_block(n);
  const int j0 = min(n, tid * B), j1 = min(n, j0 + B);
  const char* __restrict__ P = static_cast<const char*>(Pv);
  const size_t row_stride = (size_t)ld * EB;

  for (int q = tid; q < (int)rw_flag_bytes(n); q += kRwThreads) flags[q] = 0;
  if (tid == 0) mbar_init(sbar, 1u);
  int cur = start_city(key, it, (uint32_t)k, n);
  __syncthreads();
  if (tid == 0) {
    flags[cur] = 1;
    tour[0] = cur;
  }
  uint32_t phase = 0u;
  for (int t = 1; t < n; ++t) {
    if (tid == 0) bulk_load(srow, P + (size_t)cur * row_stride, row_bytes, sbar);
    const bool landed = mbar_wait(sbar, phase, polls);
    phase ^= 1u;
    if (__syncthreads_or(!landed)) {  // the wait ran out: report, let the copy land, stop
      if (tid == 0 && err) atomicExch(err, kErrTimeout);
      mbar_wait(sbar, phase ^ 1u, kRwSpin);
      return;
    }
    // pass 1: the largest unvisited value; the lowest unvisited column
    uint32_t mx = 0u;
    int first = 0x7FFFFFFF;
    for (int j = j0; j < j1; j += 4) {
      const uint32_t f = *reinterpret_cast<const volatile uint32_t*>(flags + j);
      uint32_t b[4];
      rw_bits4<PREC>(sbase, j, b);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (j + i >= j1 || ((f >> (8 * i)) & 0xFFu)) continue;
        first = min(first, j + i);
        mx = max(mx, b[i]);
      }
    }
    mx = __reduce_max_sync(ACO_FULL_MASK, mx);
    first = (int)__reduce_min_sync(ACO_FULL_MASK, (uint32_t)first);
    if (lane == 0) {
      wmax[warp] = mx;
      wfirst[warp] = first;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      mx = max(mx, wmax[w]);
      first = min(first, wfirst[w]);
    }
    int next;
    if (mx == 0u) {
      next = first < n ? first : -1;  // every unvisited value is 0
    } else {
      const int e = rw_exponent(mx);
      // pass 2: this thread's sum of quanta, then a block-wide exclusive scan
      uint64_t s = 0ull;
      for (int j = j0; j < j1; j += 4) {
        const uint32_t f = *reinterpret_cast<const volatile uint32_t*>(flags + j);
        uint32_t b[4];
        rw_bits4<PREC>(sbase, j, b);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (j + i < j1 && !((f >> (8 * i)) & 0xFFu)) s += rw_quantum(b[i], e);
      }
      uint64_t inc = s;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint64_t v = shfl_up_u64(inc, off);
        if (lane >= off) inc += v;
      }
      if (lane == 31) wsum[warp] = inc;
      __syncthreads();
      uint64_t below = 0ull, S = 0ull;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint64_t x = wsum[w];
        if (w < warp) below += x;
        S += x;
      }
      const uint64_t incl = below + inc, excl = incl - s;
      const uint4 x = philox(make_uint4(1u << 30, (uint32_t)t, (uint32_t)k, it), key);
      const uint64_t u = ((uint64_t)x.x << 32) | (uint64_t)x.y;
      const uint64_t v = __umul64hi(u, S);
      if (excl <= v && v < incl) {  // exactly one thread: the ranges partition [0, S)
        uint64_t run = excl;
        int pick = -1;
        for (int j = j0; j < j1 && pick < 0; j += 4) {
          const uint32_t f = *reinterpret_cast<const volatile uint32_t*>(flags + j);
          uint32_t b[4];
          rw_bits4<PREC>(sbase, j, b);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (pick >= 0 || j + i >= j1 || ((f >> (8 * i)) & 0xFFu)) continue;
            run += rw_quantum(b[i], e);
            if (run > v) pick = j + i;
          }
        }
        *spick = pick;
      }
      __syncthreads();
      next = *spick;
    }
    if (next < 0 || next >= n) {  // cannot happen for valid input
      if (tid == 0 && err) atomicExch(err, kErrConstruct);
      break;
    }
    if (tid == 0) {
      flags[next] = 1;
      tour[t] = next;
    }
    cur = next;
    __syncthreads();  // the flag is set, and every read of the staged row and the sums is done
  }
}

template <int PREC>
__global__ void __launch_bounds__(kRwThreads) construct_rw_kernel(const void* __restrict__ Pv, int n, int ld, int m,
                                                                  uint2 key, uint32_t it_arg,
                                                                  const uint32_t* __restrict__ it_dev,
                                                                  int32_t* __restrict__ tours,
                                                                  int32_t* __restrict__ err, uint32_t polls) {
  extern __shared__ __align__(16) uint4 rsm[];
  const int k = blockIdx.x;
  if (k >= m) return;
  const uint32_t it = it_dev ? *it_dev : it_arg;
  rw_ant<PREC>(Pv, n, ld, key, it, k, tours + (size_t)k * n, err, polls, rsm);
}

// Multi-instance form: one CTA per ant of the `count` roulette-wheel
// instances in `insts`; ant_off holds the exclusive prefix sums of their ant
// counts (ant_off[count] = the grid size).
template <int PREC>
__global__ void __launch_bounds__(kRwThreads) batch_construct_rw_kernel(const InstDev* __restrict__ insts,
                                                                        const int* __restrict__ ant_off, int count,
                                                                        int32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint4 rsm[];
  const int i = find_instance(ant_off, count, (int)blockIdx.x);
  const InstDev& I = insts[i];
  const int k = (int)blockIdx.x - __ldg(ant_off + i);
  if (!I.rw || k >= I.m) return;  // cannot happen for consistent tables
  rw_ant<PREC>(I.P, I.n, I.ld, I.key, *I.it, k, I.tours + (size_t)k * I.n, err, kRwSpin, rsm);
}

}  // namespace

int launch_construct_rw(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                        const uint32_t* it_dev, int32_t* tours, int32_t* err, uint32_t polls, cudaStream_t st) {
  if (n > kRwMaxN) return set_error(ACO_ERR_UNSUPPORTED, "roulette-wheel construction serves n <= %d", kRwMaxN);
  const int eb = prec == ACO_FP32 ? 4 : 2;
  const size_t smem = rw_smem_bytes(n, eb);
  switch (prec) {
    case ACO_FP32:
      construct_rw_kernel<ACO_FP32><<<m, kRwThreads, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, polls);
      break;
    case ACO_BF16:
      construct_rw_kernel<ACO_BF16><<<m, kRwThreads, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, polls);
      break;
    case ACO_FP16:
      construct_rw_kernel<ACO_FP16><<<m, kRwThreads, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, polls);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "construct_rw_kernel launch");
}

int launch_batch_construct_rw(const InstDev* insts, const int* ant_off, int count, int total, int32_t* err,
                              int prec, int max_n, cudaStream_t st) {
  if (count <= 0 || total <= 0) return ACO_OK;
  if (max_n > kRwMaxN) return set_error(ACO_ERR_UNSUPPORTED, "roulette-wheel construction serves n <= %d", kRwMaxN);
  const size_t smem = rw_smem_bytes(max_n, prec == ACO_FP32 ? 4 : 2);
  switch (prec) {
    case ACO_FP32:
      batch_construct_rw_kernel<ACO_FP32><<<total, kRwThreads, smem, st>>>(insts, ant_off, count, err);
      break;
    case ACO_BF16:
      batch_construct_rw_kernel<ACO_BF16><<<total, kRwThreads, smem, st>>>(insts, ant_off, count, err);
      break;
    case ACO_FP16:
      batch_construct_rw_kernel<ACO_FP16><<<total, kRwThreads, smem, st>>>(insts, ant_off, count, err);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "batch_construct_rw_kernel launch");
}

int prepare_construct_rw() {
  const int most = (int)rw_smem_bytes(kRwMaxN, 4);
  const void* fns[] = {(const void*)construct_rw_kernel<ACO_FP32>,       (const void*)construct_rw_kernel<ACO_BF16>,
                       (const void*)construct_rw_kernel<ACO_FP16>,       (const void*)batch_construct_rw_kernel<ACO_FP32>,
                       (const void*)batch_construct_rw_kernel<ACO_BF16>, (const void*)batch_construct_rw_kernel<ACO_FP16>};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(rw)");
  }
  return ACO_OK;
}

}  // namespace aco
