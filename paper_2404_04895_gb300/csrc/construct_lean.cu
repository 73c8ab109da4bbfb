// Instantiations and launchers of the lean (candidate-list) construction kernels.
#include "construct_lean.cuh"
#include "internal.h"

namespace aco {

namespace {

template <int PREC, bool FULL0, bool LISTS>
void launch_lean(int grid, size_t smem, cudaStream_t st, const void* P, int n, int ld, int m, uint2 key,
                 uint32_t it, const uint32_t* it_dev, int32_t* tours, int32_t* err, const uint2* lists,
                 const int* lcnt, const uint32_t* lkey) {
  construct_lean_kernel<PREC, FULL0, LISTS><<<grid, 32, smem, st>>>(P, n, ld, m, key, it, it_dev, tours, err, lists,
                                                                    lcnt, lkey);
}

// the lean kernel for this precision: lists and a full first round, lists
// only, or compact scans only
template <int PREC>
void launch_lean_for(bool lists, bool full0, int grid, size_t smem, cudaStream_t st, const void* P, int n, int ld,
                     int m, uint2 key, uint32_t it, const uint32_t* it_dev, int32_t* tours, int32_t* err,
                     const uint2* L, const int* lcnt, const uint32_t* lkey) {
  if (!lists)
    launch_lean<PREC, false, false>(grid, smem, st, P, n, ld, m, key, it, it_dev, tours, err, L, lcnt, lkey);
  else if (full0)
    launch_lean<PREC, true, true>(grid, smem, st, P, n, ld, m, key, it, it_dev, tours, err, L, lcnt, lkey);
  else
    launch_lean<PREC, false, true>(grid, smem, st, P, n, ld, m, key, it, it_dev, tours, err, L, lcnt, lkey);
}

template <int PREC, bool FULL0>
cudaError_t launch_batch_lean(int grid, size_t smem, cudaStream_t st, const InstDev* insts, const int* ant_off,
                              int count, int total, int* counter, int32_t* err, int max_n, int num_sms) {
  int blocks = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_construct_lean_kernel<PREC, FULL0>, 32, smem);
  if (e != cudaSuccess) return e;
  grid = (blocks < 1 ? 1 : blocks) * num_sms;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  batch_construct_lean_kernel<PREC, FULL0><<<grid, 32, smem, st>>>(insts, ant_off, count, total, counter, err, max_n);
  return cudaGetLastError();
}

template <int PREC>
void launch_probe(size_t smem, cudaStream_t st, const void* P, int n, int ld, int m, uint2 key, uint32_t it,
                  int32_t* tours, int32_t* err, const uint2* lists, const uint32_t* lkey, int probe_ant,
                  uint32_t* probe) {
  construct_lean_probe_kernel<PREC><<<m, 32, smem, st>>>(P, n, ld, m, key, it, tours, err, lists, lkey, probe_ant,
                                                         probe);
}

template <int PREC, bool FULL0>
cudaError_t allow_smem(int most) {
  cudaError_t e = cudaFuncSetAttribute(construct_lean_kernel<PREC, FULL0, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess && !FULL0)
    e = cudaFuncSetAttribute(construct_lean_kernel<PREC, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_construct_lean_kernel<PREC, FULL0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             most);
  if (e == cudaSuccess && FULL0)
    e = cudaFuncSetAttribute(construct_lean_probe_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  return e;
}

}  // namespace

int launch_construct_lean(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                          const uint32_t* it_dev, int32_t* tours, int32_t* err, const uint2* lists,
                          const int* lcnt, const uint32_t* lkey, cudaStream_t st) {
  const int eb = prec == ACO_FP32 ? 4 : 2;
  if (n > lean_max_n(eb)) return set_error(ACO_ERR_UNSUPPORTED, "lean construction serves n <= %d", lean_max_n(eb));
  const size_t smem = lean_smem_bytes(n, eb, kLeanAnts);
  const int grid = (m + kLeanAnts - 1) / kLeanAnts;
  const bool full0 = n >= 32;  // every list then has >= 32 entries
  const bool has_lists = lists != nullptr;
  switch (prec) {
    case ACO_FP32:
      launch_lean_for<ACO_FP32>(has_lists, full0, grid, smem, st, P, n, ld, m, key, it, it_dev, tours, err, lists,
                                lcnt, lkey);
      break;
    case ACO_BF16:
      launch_lean_for<ACO_BF16>(has_lists, full0, grid, smem, st, P, n, ld, m, key, it, it_dev, tours, err, lists,
                                lcnt, lkey);
      break;
    case ACO_FP16:
      launch_lean_for<ACO_FP16>(has_lists, full0, grid, smem, st, P, n, ld, m, key, it, it_dev, tours, err, lists,
                                lcnt, lkey);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "construct_lean_kernel launch");
}

int launch_batch_construct_lean(const InstDev* insts, const int* ant_off, int count, int total,
                                int* counter, int32_t* err, int prec, int min_n, int max_n, int num_sms,
                                cudaStream_t st) {
  const int eb = prec == ACO_FP32 ? 4 : 2;
  if (max_n > lean_max_n(eb)) return set_error(ACO_ERR_UNSUPPORTED, "lean construction serves n <= %d", lean_max_n(eb));
  const size_t smem = lean_smem_bytes(max_n, eb);
  const bool full0 = min_n >= 32;
  cudaError_t e;
  switch (prec) {
    case ACO_FP32:
      e = (full0 ? launch_batch_lean<ACO_FP32, true> : launch_batch_lean<ACO_FP32, false>)(
          0, smem, st, insts, ant_off, count, total, counter, err, max_n, num_sms);
      break;
    case ACO_BF16:
      e = (full0 ? launch_batch_lean<ACO_BF16, true> : launch_batch_lean<ACO_BF16, false>)(
          0, smem, st, insts, ant_off, count, total, counter, err, max_n, num_sms);
      break;
    default:
      e = (full0 ? launch_batch_lean<ACO_FP16, true> : launch_batch_lean<ACO_FP16, false>)(
          0, smem, st, insts, ant_off, count, total, counter, err, max_n, num_sms);
  }
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "batch_construct_lean_kernel launch");
}

int prepare_construct_lean() {
  const int most = (int)lean_smem_bytes(lean_max_n(4), 4, kLeanAnts);
  cudaError_t e = allow_smem<ACO_FP32, false>(most);
  if (e == cudaSuccess) e = allow_smem<ACO_FP32, true>(most);
  if (e == cudaSuccess) e = allow_smem<ACO_BF16, false>(most);
  if (e == cudaSuccess) e = allow_smem<ACO_BF16, true>(most);
  if (e == cudaSuccess) e = allow_smem<ACO_FP16, false>(most);
  if (e == cudaSuccess) e = allow_smem<ACO_FP16, true>(most);
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "cudaFuncSetAttribute(lean)");
}

}  // namespace aco

using namespace aco;

extern "C" int aco_op_construct_probe(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                                      int32_t* tours_dev, int32_t* err_dev, const void* lists_dev,
                                      const uint32_t* lkey_dev, int probe_ant, uint32_t* probe_dev, void* stream) {
  if (!P_dev || !tours_dev || !lists_dev || !lkey_dev || !probe_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (n < 32 || n > kLeanMaxN) return set_error(ACO_ERR_ARG, "the probed construction serves 32 <= n <= %d", kLeanMaxN);
  if (ld < n || (ld & 7) || !aligned16(P_dev)) return set_error(ACO_ERR_ARG, "P: ld >= n, a multiple of 8, 16-byte aligned");
  if (m < 1 || m > ACO_MAX_M || probe_ant < 0 || probe_ant >= m) return set_error(ACO_ERR_ARG, "m or probe_ant out of range");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  int rc = prepare_kernels();
  if (rc) return rc;
  const int eb = prec == ACO_FP32 ? 4 : 2;
  const size_t smem = lean_smem_bytes(n, eb, 1);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint2* L = static_cast<const uint2*>(lists_dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == ACO_FP32)
    launch_probe<ACO_FP32>(smem, st, P_dev, n, ld, m, key, it, tours_dev, err_dev, L, lkey_dev, probe_ant, probe_dev);
  else if (prec == ACO_BF16)
    launch_probe<ACO_BF16>(smem, st, P_dev, n, ld, m, key, it, tours_dev, err_dev, L, lkey_dev, probe_ant, probe_dev);
  else
    launch_probe<ACO_FP16>(smem, st, P_dev, n, ld, m, key, it, tours_dev, err_dev, L, lkey_dev, probe_ant, probe_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, "construct_lean_probe_kernel launch");
}
