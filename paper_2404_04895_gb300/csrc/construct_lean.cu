// Instantiations and launchers of the lean (candidate-list) construction kernels.
#include "construct_lean.cuh"
#include "internal.h"

namespace aco {

int launch_construct_lean(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                          const uint32_t* it_dev, int32_t* tours, int32_t* err, const uint2* lists,
                          const int* lcnt, const uint32_t* lkey, cudaStream_t st) {
  const int eb = prec == ACO_FP32 ? 4 : 2;
  if (n > lean_max_n(eb)) return set_error(ACO_ERR_UNSUPPORTED, "lean construction serves n <= %d", lean_max_n(eb));
  const size_t smem = lean_smem_bytes(n, eb, kLeanAnts);
  const int grid = (m + kLeanAnts - 1) / kLeanAnts;
  switch (prec) {
    case ACO_FP32:
      construct_lean_kernel<ACO_FP32><<<grid, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, lists,
                                                              lcnt, lkey);
      break;
    case ACO_BF16:
      construct_lean_kernel<ACO_BF16><<<grid, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, lists,
                                                              lcnt, lkey);
      break;
    case ACO_FP16:
      construct_lean_kernel<ACO_FP16><<<grid, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, lists,
                                                              lcnt, lkey);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "construct_lean_kernel launch");
}

int launch_batch_construct_lean(const InstDev* insts, const int* ant_off, int count, int total,
                                int* counter, int32_t* err, int prec, int max_n, int num_sms,
                                cudaStream_t st) {
  const int eb = prec == ACO_FP32 ? 4 : 2;
  if (max_n > lean_max_n(eb)) return set_error(ACO_ERR_UNSUPPORTED, "lean construction serves n <= %d", lean_max_n(eb));
  const size_t smem = lean_smem_bytes(max_n, eb);
  int blocks = 0;
  cudaError_t e = cudaSuccess;
  switch (prec) {
    case ACO_FP32:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_construct_lean_kernel<ACO_FP32>, 32, smem);
      break;
    case ACO_BF16:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_construct_lean_kernel<ACO_BF16>, 32, smem);
      break;
    default:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_construct_lean_kernel<ACO_FP16>, 32, smem);
  }
  if (e != cudaSuccess) return cuda_error(e, "occupancy query (lean)");
  int grid = (blocks < 1 ? 1 : blocks) * num_sms;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  switch (prec) {
    case ACO_FP32:
      batch_construct_lean_kernel<ACO_FP32><<<grid, 32, smem, st>>>(insts, ant_off, count, total, counter, err, max_n);
      break;
    case ACO_BF16:
      batch_construct_lean_kernel<ACO_BF16><<<grid, 32, smem, st>>>(insts, ant_off, count, total, counter, err, max_n);
      break;
    default:
      batch_construct_lean_kernel<ACO_FP16><<<grid, 32, smem, st>>>(insts, ant_off, count, total, counter, err, max_n);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "batch_construct_lean_kernel launch");
}

int prepare_construct_lean() {
  const int most = (int)lean_smem_bytes(lean_max_n(4), 4, kLeanAnts);
  cudaError_t e = cudaFuncSetAttribute(construct_lean_kernel<ACO_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(construct_lean_kernel<ACO_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(construct_lean_kernel<ACO_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_construct_lean_kernel<ACO_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_construct_lean_kernel<ACO_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_construct_lean_kernel<ACO_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "cudaFuncSetAttribute(lean)");
}

}  // namespace aco
