// Selection frequencies of independent roulette on one row (the Bernoulli
// trials of the paper's AdaIR visualisation, Sec. 3.3.1 / Fig. 4).
//
// Trial tr draws r_j for every candidate j from Philox4x32-10 with counter
// (j >> 2, tr mod 2^32, tr div 2^32, salt), word j & 3, r = ((x >> 8) | 1)
// 2^-24, and picks argmax over the unvisited j of fl32(r_j * q_j), lowest j
// on ties -- the selection step of Sec. 2.4 on the row q (for AdaIR, q is
// the row raised to 1/gamma, as the path computes it).  counts[j] += the
// number of trials j wins.  One thread per trial (grid-stride); the counts
// are gathered in a shared-memory histogram per CTA.
#include "common.cuh"
#include "internal.h"

namespace aco {

namespace {

constexpr int kStudyMaxN = 4096;

__global__ void __launch_bounds__(256) selection_counts_kernel(const float* __restrict__ q,
                                                               const uint8_t* __restrict__ visited, int n,
                                                               unsigned long long trials, uint2 key,
                                                               uint32_t salt,
                                                               unsigned long long* __restrict__ counts) {
  __shared__ unsigned int hist[kStudyMaxN];
  for (int j = threadIdx.x; j < n; j += blockDim.x) hist[j] = 0u;
  __syncthreads();
  const PhiloxKeys ks = philox_keys(key);
  for (unsigned long long tr = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; tr < trials;
       tr += (unsigned long long)gridDim.x * blockDim.x) {
    float bs = -1.0f;
    int bj = -1;
    for (int j0 = 0; j0 < n; j0 += 4) {
      const uint4 x = philox(make_uint4((uint32_t)(j0 >> 2), (uint32_t)tr, (uint32_t)(tr >> 32), salt), ks);
      const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = j0 + i;
        if (j >= n || (visited && visited[j])) continue;
        const float s = __fmul_rn(uniform01(w[i]), __ldg(q + j));
        if (bj < 0 || s > bs) {  // ascending j: equal scores keep the lower j
          bs = s;
          bj = j;
        }
      }
    }
    if (bj >= 0) atomicAdd(hist + bj, 1u);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (hist[j]) atomicAdd(counts + j, (unsigned long long)hist[j]);
}

}  // namespace

}  // namespace aco

using namespace aco;

extern "C" int aco_op_selection_counts(const float* q_dev, const uint8_t* visited_dev, int n,
                                       unsigned long long trials, uint64_t seed, uint32_t salt,
                                       unsigned long long* counts_dev, void* stream) {
  if (!q_dev || !counts_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (n < 1 || n > kStudyMaxN) return set_error(ACO_ERR_ARG, "n=%d outside [1, %d]", n, kStudyMaxN);
  if (trials == 0) return ACO_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long want = (trials + 255) / 256;
  const unsigned long long cap = (unsigned long long)(sms > 0 ? sms : 1) * 8;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  selection_counts_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      q_dev, visited_dev, n, trials, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), salt, counts_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "selection_counts_kernel launch");
}
