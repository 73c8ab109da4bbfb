// Allocation-free variant of the tour-length + deterministic deposit pair.
//
// Some callers cannot allocate device memory at the point where they update
// pheromone: embedders whose device memory all belongs to a framework's pool
// or to a budget fixed at start-up, which they may not go around, and loops
// with a latency bound, where a cudaMalloc (which may synchronise the device
// and has no bounded running time) is not allowed.  aco_op_tour_length +
// aco_op_deposit need a scratch buffer for the index mapping (2*n*m int32) and
// the weights Q/L (m fp64) that such callers would otherwise have to
// allocate.  This entry point keeps that scratch in a fixed, file-scope device
// array instead; the caller still passes every input and output.
//
// The array is part of this library's device image: every GPU that loads the
// library holds its ACO_NOALLOC_SCRATCH_BYTES until the process exits.  All
// calls share it and it keeps the last call's contents, so calls that overlap
// on the GPU (different streams, threads or processes sharing a context) race;
// serialise them.  Each call clears the index mapping before filling it, so
// an entry a malformed tour leaves unwritten is never one an earlier call
// wrote; the weights are written in full before they are read.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "internal.h"

namespace aco {

static __device__ __align__(256) unsigned char g_noalloc_scratch[ACO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (host code only ever sees a host-side stand-in for the symbol).
static int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  ACO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(ACO_ERR_UNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return ACO_OK;
}

static size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace aco

using namespace aco;

extern "C" int aco_op_deposit_tours_noalloc(float* tau_dev, int n, int ld, const double* D_dev,
                                            const int32_t* tours_dev, int m, float rho, float Q,
                                            double* L_dev, int32_t* err_dev, void* stream) {
  if (!tau_dev || !D_dev || !tours_dev || !L_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (n < 3 || n > ACO_MAX_N || m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "n or m out of range");
  if (ld < n || (ld & 7) || !aligned16(tau_dev))
    return set_error(ACO_ERR_ARG, "tau: ld must be >= n and a multiple of 8, base 16-byte aligned");
  if (!(rho >= 0.0f && rho <= 1.0f)) return set_error(ACO_ERR_ARG, "rho outside [0, 1]");
  if (!(Q > 0.0f) || !std::isfinite(Q)) return set_error(ACO_ERR_ARG, "Q must be finite and > 0");
  const size_t c_bytes = round256((size_t)m * sizeof(double));
  const size_t nbr_bytes = (size_t)n * m * 2 * sizeof(int32_t);
  const size_t need = c_bytes + nbr_bytes;
  if (need > ACO_NOALLOC_SCRATCH_BYTES)
    return set_error(ACO_ERR_ARG,
                     "n=%d, m=%d need %zu scratch bytes; the allocation-free deposit holds %zu "
                     "(8*m + 8*n*m must fit)", n, m, need, (size_t)ACO_NOALLOC_SCRATCH_BYTES);
  int rc = prepare_kernels();
  if (rc) return rc;
  unsigned char* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  double* c = reinterpret_cast<double*>(scratch);
  int32_t* nbr = reinterpret_cast<int32_t*>(scratch + c_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // -1 everywhere: an entry no tour writes is skipped by the deposit
  ACO_CUDA_TRY(cudaMemsetAsync(nbr, 0xFF, nbr_bytes, st));
  rc = launch_tour_length(D_dev, n, tours_dev, m, Q, L_dev, c, nbr, false, st);
  if (rc) return rc;
  return launch_deposit(tau_dev, ACO_FP32, n, ld, nbr, c, m, rho, nullptr, err_dev, st);
}
