// Measurement kernels for the construction step's roofline ceilings.  They
// compute nothing of the method; they time the three resources a step of
// Sec. 2.4 draws on, in the form the construction kernels use them:
//   row reads   warps reading whole random rows of an M_p-sized buffer with
//               16-byte coalesced loads (the full scan's traffic): bytes/s of
//               the memory level that holds the buffer (L2 for 50-100 MB,
//               HBM beyond it)
//   philox      Philox4x32-10 blocks mapped to four scored candidates each,
//               fl32(r * p) and a running argmax (the scan's arithmetic):
//               candidates/s of the SMs' ALUs
//   chase       one warp per SM following a random cycle of dependent loads
//               through a buffer (a step's critical path when the next row is
//               not already in flight): cycles per dependent load
// Every kernel writes a checksum so that the compiler keeps its work; the
// buffers are the caller's.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace aco {

namespace {

// a 32-bit mix (the finaliser of MurmurHash3) for picking rows
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// Warp w reads rows_per_warp rows r = mix(w, i) mod rows, each row_bytes long
// (a multiple of 16), lane l taking 16-byte chunks l, l + 32, ...; eight
// chunks per lane in flight.
__global__ void __launch_bounds__(256) row_reads_kernel(const uint4* __restrict__ buf, size_t rows,
                                                        int row_chunks, int rows_per_warp, uint32_t salt,
                                                        unsigned long long* __restrict__ sink) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  uint32_t acc = 0u;
  for (int i = 0; i < rows_per_warp; ++i) {
    const size_t r = (size_t)mix32(w * 0x9E3779B9u + (uint32_t)i * 0x7F4A7C15u + salt) % rows;
    const uint4* row = buf + r * (size_t)row_chunks;
    for (int c0 = lane; c0 < row_chunks; c0 += 8 * 32) {
      uint4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + 32 * u;
        v[u] = c < row_chunks ? __ldcg(row + c) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
  }
  acc = __reduce_xor_sync(ACO_FULL_MASK, acc);
  if (lane == 0) atomicAdd(sink, (unsigned long long)acc);
}

// Thread g scores blocks_per_thread Philox blocks of counter (b, g, salt, 7):
// four candidates each, score fl32(r * p) with r the construction's uniform
// and p a fixed value, kept as a running argmax (lowest index on ties).
__global__ void __launch_bounds__(256) philox_scores_kernel(uint2 key, int blocks_per_thread, uint32_t salt,
                                                            float p, unsigned long long* __restrict__ sink) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  const PhiloxKeys ks = philox_keys(key);
  float best = -1.0f;
  uint32_t best_j = 0u;
  for (int b = 0; b < blocks_per_thread; ++b) {
    const uint4 x = philox(make_uint4((uint32_t)b, g, salt, 7u), ks);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float s = __fmul_rn(uniform01(w[i]), p);
      const uint32_t j = 4u * (uint32_t)b + (uint32_t)i;
      if (s > best) {
        best = s;
        best_j = j;
      }
    }
  }
  const uint32_t h = __reduce_xor_sync(ACO_FULL_MASK, __float_as_uint(best) ^ best_j);
  if ((threadIdx.x & 31) == 0) atomicAdd(sink, (unsigned long long)h);
}

// One thread per CTA follows next[] from slot blockIdx.x for `hops` dependent
// loads; out_cycles[blockIdx.x] = clock64 cycles per load.
__global__ void chase_kernel(const uint32_t* __restrict__ next, int hops, unsigned long long* __restrict__ out_cycles,
                             unsigned long long* __restrict__ sink) {
  if (threadIdx.x != 0) return;
  uint32_t at = blockIdx.x * 977u;
  at = __ldcg(next + at);  // the first load is outside the timed chain
  const long long t0 = clock64();
  for (int h = 0; h < hops; ++h) at = __ldcg(next + at);
  const long long t1 = clock64();
  out_cycles[blockIdx.x] = (unsigned long long)((t1 - t0) / (hops > 0 ? hops : 1));
  atomicAdd(sink, (unsigned long long)at);
}

}  // namespace

}  // namespace aco

using namespace aco;

extern "C" {

int aco_ceiling_row_reads(const void* buf_dev, size_t bytes, int row_bytes, int warps, int rows_per_warp,
                          uint32_t salt, unsigned long long* sink_dev, void* stream) {
  if (!buf_dev || !sink_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (!aligned16(buf_dev)) return set_error(ACO_ERR_ARG, "buffer must be 16-byte aligned");
  if (row_bytes < 16 || (row_bytes & 15) || bytes < (size_t)row_bytes)
    return set_error(ACO_ERR_ARG, "row_bytes must be a multiple of 16 and at most the buffer size");
  if (warps < 8 || (warps & 7) || rows_per_warp < 1)
    return set_error(ACO_ERR_ARG, "warps must be a positive multiple of 8, rows_per_warp >= 1");
  const size_t rows = bytes / (size_t)row_bytes;
  row_reads_kernel<<<warps / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const uint4*>(buf_dev), rows, row_bytes / 16, rows_per_warp, salt, sink_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "row_reads_kernel");
}

int aco_ceiling_philox(uint64_t seed, int threads, int blocks_per_thread, uint32_t salt,
                       unsigned long long* sink_dev, void* stream) {
  if (!sink_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (threads < 256 || (threads & 255) || blocks_per_thread < 1)
    return set_error(ACO_ERR_ARG, "threads must be a positive multiple of 256, blocks_per_thread >= 1");
  philox_scores_kernel<<<threads / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), blocks_per_thread, salt, 0.75f, sink_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "philox_scores_kernel");
}

int aco_ceiling_chase(const uint32_t* next_dev, size_t slots, int chains, int hops,
                      unsigned long long* cycles_dev, unsigned long long* sink_dev, void* stream) {
  if (!next_dev || !cycles_dev || !sink_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (chains < 1 || hops < 1 || slots < (size_t)chains * 977u + 1u || slots > 0xFFFFFFFFull)
    return set_error(ACO_ERR_ARG, "chains, hops >= 1 and 977 * chains < slots < 2^32");
  chase_kernel<<<chains, 32, 0, static_cast<cudaStream_t>(stream)>>>(next_dev, hops, cycles_dev, sink_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "chase_kernel");
}

}  // extern "C"
