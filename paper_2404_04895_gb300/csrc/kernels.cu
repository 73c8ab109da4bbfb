// The non-construction kernels of one TensorACO iteration (sm_103a):
//   heuristic   Sec. 2.1: fp64 distances and eta^beta           (once per instance)
//   build_P     Eq. 1:   M_p = tau^alpha * eta^beta [^(1/gamma)] (per iteration)
//   tour_length Eq. 3:   f(s) exact, rounded once to fp64; Q/f; the index mapping of Eq. 2
//   best        iteration best merged into the running best
//   deposit     Sec. 2.3: evaporation + Delta M_tau (deterministic / atomic)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "steps.cuh"

namespace aco {

// ---------------------------------------------------------------------------
// Sec. 2.1: D_ij = sqrt(dx^2 + dy^2) (fp64), H_ij = fl32((1/max(d,1e-9))^beta),
// H_ii = 0, H zero in the padding columns n <= j < ld.  Both are symmetric
// bit for bit: x_j - x_i is exactly -(x_i - x_j) (rounding to nearest is
// symmetric) and squaring drops the sign.  So one CTA takes a 32 x 32 tile
// (I, J) with I <= J, computes each entry once (1/d by the correctly rounded
// reciprocal, the same value as a correctly rounded 1.0 / d), writes it
// row-wise at (i, j) and, through shared memory, row-wise at (j, i).
// PACKED: D is the strictly upper triangle (tri_index), written at (i, j),
// i < j, only.  Grid (T, T), T = ceil(n / 32); blocks with I > J return at
// once.
// ---------------------------------------------------------------------------
template <bool PACKED>
__global__ void __launch_bounds__(256) heuristic_kernel(const float* __restrict__ xy, int n, int beta,
                                                        double* __restrict__ D, float* __restrict__ H, int ld) {
  __shared__ double sd[32][33];
  __shared__ float sh[32][33];
  const int I = blockIdx.y, J = blockIdx.x;
  if (I > J) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = 32 * J + tx;
  double xj = 0.0, yj = 0.0;
  if (j < n) {
    xj = (double)xy[2 * j];
    yj = (double)xy[2 * j + 1];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = ty + 8 * k, i = 32 * I + r;
    double d = 0.0;
    float h = 0.0f;
    if (i < n && j < n) {
      const double dx = __dsub_rn((double)xy[2 * i], xj);
      const double dy = __dsub_rn((double)xy[2 * i + 1], yj);
      d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
      if (i != j) h = __double2float_rn(powi_f64(__drcp_rn(d > 1e-9 ? d : 1e-9), beta));
      if (D) {
        if (!PACKED)
          D[(size_t)i * n + j] = d;
        else if (i < j)
          D[tri_index(n, i, j)] = d;
      }
      H[(size_t)i * ld + j] = h;
    }
    sd[r][tx] = d;
    sh[r][tx] = h;
    if (J == (int)gridDim.x - 1 && i < n)  // this row's padding columns
      for (int c = n + tx; c < ld; c += 32) H[(size_t)i * ld + c] = 0.0f;
  }
  if (I == J) return;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = ty + 8 * k;  // row 32J + r of the mirrored tile, column 32I + tx
    const int jr = 32 * J + r, ic = 32 * I + tx;
    if (jr < n && ic < n) {
      if (D && !PACKED) D[(size_t)jr * n + ic] = sd[tx][r];
      H[(size_t)jr * ld + ic] = sh[tx][r];
    }
  }
}

__global__ void fill_u16_kernel(unsigned short* __restrict__ a, size_t count, unsigned short v) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (size_t)gridDim.x * blockDim.x)
    a[q] = v;
}

__global__ void fill_kernel(float* __restrict__ a, size_t count, float v) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (size_t)gridDim.x * blockDim.x)
    a[q] = v;
}

// ---------------------------------------------------------------------------
// Single-instance wrappers around the device functions of steps.cuh.
// ---------------------------------------------------------------------------
template <int PREC, bool TB>
__global__ void __launch_bounds__(256) build_P_kernel(const void* __restrict__ tau,
                                                      const float* __restrict__ H, int n, int ld,
                                                      int alpha, float inv_gamma_arg,
                                                      const float* __restrict__ inv_gamma_dev,
                                                      const uint32_t* __restrict__ it_dev,
                                                      int n_sched, void* __restrict__ Pv) {
  __shared__ float red[32];
  const int i = blockIdx.x;
  float inv_gamma = inv_gamma_arg;
  if (inv_gamma_dev) {
    const uint32_t it = *it_dev;
    inv_gamma = inv_gamma_dev[it < (uint32_t)n_sched ? it : (uint32_t)(n_sched - 1)];
  }
  const size_t eb = PREC == ACO_FP32 ? 4 : 2;
  build_P_row<PREC, TB>(static_cast<const char*>(tau) + (size_t)i * ld * (TB ? 2 : 4), H + (size_t)i * ld, n,
                        ld, i, alpha, inv_gamma, static_cast<char*>(Pv) + (size_t)i * ld * eb, red);
}

template <int PREC>
__global__ void __launch_bounds__(256) build_lists_kernel(const void* __restrict__ Pv, int n, int ld,
                                                          uint2* __restrict__ lists,
                                                          int* __restrict__ lcnt,
                                                          uint32_t* __restrict__ lkey) {
  __shared__ uint32_t scratch[kListScratchWords];
  const int i = blockIdx.x;
  const size_t eb = PREC == ACO_FP32 ? 4 : 2;
  build_list_row<PREC>(static_cast<const char*>(Pv) + (size_t)i * ld * eb, n,
                       lists + (size_t)i * kListMax, lcnt + i, lkey + i, scratch);
}

// Eq. 1 and the candidate list of row i in one pass; the list's collection
// threshold comes from the row's previous bound (lkey, rewritten here) and
// the evaporation keep^alpha, AdaIR's exponent from the schedule.
template <int PREC, bool TB>
__global__ void __launch_bounds__(256, 6) build_P_lists_kernel(const void* __restrict__ tau, const float* __restrict__ H,
                                                            int n, int ld, int alpha, float inv_gamma_arg,
                                                            const float* __restrict__ inv_gamma_dev,
                                                            const uint32_t* __restrict__ it_dev, int n_sched,
                                                            float keep, void* __restrict__ Pv, uint2* __restrict__ lists,
                                                            int* __restrict__ lcnt, uint32_t* __restrict__ lkey) {
  __shared__ uint32_t scratch[kListScratchWords];
  __shared__ float red[32];
  const int i = blockIdx.x;
  float inv_gamma = inv_gamma_arg, ig_prev = inv_gamma_arg;
  if (inv_gamma_dev) {
    const uint32_t it = *it_dev;
    const uint32_t last = (uint32_t)(n_sched - 1);
    inv_gamma = inv_gamma_dev[it < last ? it : last];
    ig_prev = it > 0u ? inv_gamma_dev[it - 1u < last ? it - 1u : last] : 0.0f;
  }
  const uint32_t guess = list_guess(lkey[i], keep, alpha, inv_gamma, ig_prev);
  const size_t eb = PREC == ACO_FP32 ? 4 : 2;
  build_P_lists_row<PREC, TB>(static_cast<const char*>(tau) + (size_t)i * ld * (TB ? 2 : 4), H + (size_t)i * ld, n, ld,
                              i, alpha, inv_gamma, static_cast<char*>(Pv) + (size_t)i * ld * eb,
                              lists + (size_t)i * kListMax, lcnt + i, lkey + i, guess, scratch, red);
}

// One CTA of W warps per ant (W = 1: 8 ants per CTA, one warp each); PACKED
// as tour_length_exact.
template <int W, bool PACKED>
__global__ void __launch_bounds__(256) tour_length_kernel(const double* __restrict__ D, int n,
                                                          const int32_t* __restrict__ tours,
                                                          int m, float Q, double* __restrict__ L,
                                                          double* __restrict__ c,
                                                          int32_t* __restrict__ nbr) {
  __shared__ unsigned long long sacc[(W == 1 ? 8 : 1) * (kLenDigits + 1)];
  const int wid = (int)(threadIdx.x >> 5);
  const int k = W == 1 ? blockIdx.x * (blockDim.x >> 5) + wid : blockIdx.x;
  if (k >= m) return;
  tour_length_exact<W, false, PACKED>(D, n, tours + (size_t)k * n, k, Q, L, c,
                       nbr ? static_cast<void*>(reinterpret_cast<int2*>(nbr) + k) : nullptr, m, W == 1 ? 0 : wid,
                       sacc + (W == 1 ? wid * (kLenDigits + 1) : 0));
}

// Two ants per CTA, W warps each.  Their index mappings are staged in shared
// memory by city, 16 bits per neighbour (filled with 0xFFFF first: a city
// missing from a tour reads as no neighbour, -1), and written out row by row,
// both ants' int2 entries of a city in one 16-byte store: half the scattered
// stores of writing every entry on its own, which dominate this step.  Ants
// 2 blockIdx.x and 2 blockIdx.x + 1; m even (rows of nbr 16-byte aligned),
// nbr 16-byte aligned,
// n <= kTourPairMaxN.  Dynamic shared memory: 8 n bytes.
template <int W, bool PACKED>
__global__ void __launch_bounds__(64 * W) tour_length_pair_kernel(const double* __restrict__ D, int n,
                                                                  const int32_t* __restrict__ tours,
                                                                  int m, float Q, double* __restrict__ L,
                                                                  double* __restrict__ c,
                                                                  int32_t* __restrict__ nbr) {
  extern __shared__ __align__(16) uint2 stage[];  // [n]: packed (pred, succ) of ant 2b, then of ant 2b + 1
  __shared__ unsigned long long sacc[2 * (kLenDigits + 1)];
  const int wid = (int)(threadIdx.x >> 5);
  const int a = wid / W;
  const int k = 2 * (int)blockIdx.x + a;
  for (int q = threadIdx.x; q < n; q += blockDim.x) stage[q] = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
  __syncthreads();
  tour_length_exact<W, true, PACKED>(D, n, tours + (size_t)k * n, k, Q, L, c, reinterpret_cast<uint32_t*>(stage) + a, 2,
                             wid - a * W, sacc + a * (kLenDigits + 1));
  __syncthreads();
  auto wide = [](uint32_t h) { return h == 0xFFFFu ? -1 : (int)h; };
  int4* out = reinterpret_cast<int4*>(nbr) + blockIdx.x;  // row q of nbr holds m / 2 int4
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const uint2 v = stage[q];
    out[(size_t)q * (m / 2)] = make_int4(wide(v.x & 0xFFFFu), wide(v.x >> 16), wide(v.y & 0xFFFFu), wide(v.y >> 16));
  }
}

__global__ void __launch_bounds__(1024) best_kernel(const double* __restrict__ L,
                                                    const int32_t* __restrict__ tours, int n,
                                                    int m, int32_t* __restrict__ best_tour,
                                                    double* __restrict__ best_len,
                                                    uint32_t* __restrict__ it_dev,
                                                    double* __restrict__ c, int topk,
                                                    int2* __restrict__ dep, int32_t* __restrict__ err) {
  __shared__ double sl[32];
  __shared__ int sk[33];
  __shared__ int sred[300];
  best_block(L, tours, n, m, best_tour, best_len, it_dev, sl, sk);
  if (c) select_topk_block(L, m, topk, c, sred);
  if (dep) {
    const int2 d = deposit_scale_block(c, m, sred);
    if (threadIdx.x == 0) {
      *dep = d;
      if (d.y == kDepBad && err) atomicExch(err, kErrDepositRange);
    }
  }
}

// One CTA per row.  The weights' scaling comes from dep (written by the best
// kernel) or, when dep is null, is derived by every CTA from c itself.
template <bool TB>
__global__ void __launch_bounds__(kDepThreads) deposit_kernel(void* __restrict__ tau, int n, int ld,
                                                              const int32_t* __restrict__ nbr,
                                                              const double* __restrict__ c, int m,
                                                              float keep, const int2* __restrict__ dep,
                                                              int cap, int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int sred[100];
  int2 d;
  if (dep) {
    d = *dep;
  } else {
    d = deposit_scale_block(c, m, sred);
    if (d.y == kDepBad && blockIdx.x == 0 && threadIdx.x == 0 && err) atomicExch(err, kErrDepositRange);
  }
  const int a = blockIdx.x;
  deposit_row_exact<TB>(static_cast<char*>(tau) + (size_t)a * ld * (TB ? 2 : 4), n,
                        reinterpret_cast<const int2*>(nbr) + (size_t)a * m, c, m, keep, d.x, d.y, cap, smem);
}

// The deterministic deposit of row a followed, in the same CTA, by the next
// iteration's M_p and candidate list of that row (build_P_lists_row) from
// the tau row just written, read back through the L2.  *it_dev is the next
// iteration's index by then (the best kernel advances it), so AdaIR's
// exponent and the list's guess are those build_P_lists_kernel would use at
// the start of that iteration; the tau row is not read from HBM a second
// time.  Dynamic shared memory: the deposit's, reused as the list scratch.
template <int PREC, bool TB>
__global__ void __launch_bounds__(kDepThreads, 6) deposit_P_lists_kernel(
    void* __restrict__ tau, int n, int ld, const int32_t* __restrict__ nbr, const double* __restrict__ c, int m,
    float keep, const int2* __restrict__ dep, int cap, const float* __restrict__ H, int alpha,
    const float* __restrict__ inv_gamma_dev, const uint32_t* __restrict__ it_dev, int n_sched,
    void* __restrict__ Pv, uint2* __restrict__ lists, int* __restrict__ lcnt, uint32_t* __restrict__ lkey) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float red[32];
  const int a = blockIdx.x;
  const int2 d = *dep;
  char* tau_row = static_cast<char*>(tau) + (size_t)a * ld * (TB ? 2 : 4);
  deposit_row_exact<TB>(tau_row, n, reinterpret_cast<const int2*>(nbr) + (size_t)a * m, c, m, keep, d.x, d.y, cap,
                        smem);  // ends with a block barrier: the row's stores are visible to the CTA
  float inv_gamma = 1.0f, ig_prev = 1.0f;
  if (inv_gamma_dev) {
    const uint32_t it = *it_dev;
    const uint32_t last = (uint32_t)(n_sched - 1);
    inv_gamma = inv_gamma_dev[it < last ? it : last];
    ig_prev = it > 0u ? inv_gamma_dev[it - 1u < last ? it - 1u : last] : 0.0f;
  }
  const uint32_t guess = list_guess(lkey[a], keep, alpha, inv_gamma, ig_prev);
  const size_t eb = PREC == ACO_FP32 ? 4 : 2;
  build_P_lists_row<PREC, TB, true>(tau_row, H + (size_t)a * ld, n, ld, a, alpha, inv_gamma,
                                    static_cast<char*>(Pv) + (size_t)a * ld * eb, lists + (size_t)a * kListMax,
                                    lcnt + a, lkey + a, guess, reinterpret_cast<uint32_t*>(smem), red);
}

// tau <- fl32(keep * tau), keep = fl32(1 - rho): evaporation in fp32
__global__ void evaporate_kernel(float* __restrict__ tau, int n, int ld, float keep) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float* p = tau + (size_t)i * ld + j;
  *p = __fmul_rn(keep, *p);
}

// Float-atomic deposit: every directed tour edge adds fl32(c_k) in hardware order.
__global__ void deposit_atomic_kernel(float* __restrict__ tau, int n, int ld,
                                      const int32_t* __restrict__ tours,
                                      const double* __restrict__ c, int m) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)m * n) return;
  const int k = (int)(q / n), t = (int)(q % n);
  const int32_t* p = tours + (size_t)k * n;
  const int a = p[t], b = p[t > 0 ? t - 1 : n - 1];
  if ((unsigned)a >= (unsigned)n || (unsigned)b >= (unsigned)n) return;
  const float cf = __double2float_rn(c[k]);
  atomicAdd(tau + (size_t)a * ld + b, cf);
  atomicAdd(tau + (size_t)b * ld + a, cf);
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, uint2 key, uint32_t* __restrict__ out,
                              int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const uint4 c = reinterpret_cast<const uint4*>(ctr)[q];
  reinterpret_cast<uint4*>(out)[q] = philox(c, key);
}

__global__ void pow_own_kernel(const float* __restrict__ x, float e, float* __restrict__ out,
                               int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count) out[q] = pow_own(x[q], e);
}

// Sec. 2.3 selection alone (step-level call): zero the weights of all but the
// k shortest paths.
__global__ void __launch_bounds__(1024) select_topk_kernel(const double* __restrict__ L, int m, int k,
                                                           double* __restrict__ c) {
  __shared__ int sred[300];
  select_topk_block(L, m, k, c, sred);
}

// ------------------------------------------------------------------ launchers
static int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, what);
}

int launch_heuristic(const float* xy, int n, int beta, double* D, float* H, int ld, bool packed,
                     cudaStream_t st) {
  const int T = (n + 31) / 32;
  dim3 grid(T, T);
  if (packed)
    heuristic_kernel<true><<<grid, 256, 0, st>>>(xy, n, beta, D, H, ld);
  else
    heuristic_kernel<false><<<grid, 256, 0, st>>>(xy, n, beta, D, H, ld);
  return check_launch("heuristic_kernel");
}

int launch_fill_tau(void* tau, int tau_prec, int n, int ld, float v, cudaStream_t st) {
  if (tau_prec != ACO_BF16) return launch_fill(static_cast<float*>(tau), n, ld, v, st);
  const size_t count = (size_t)n * ld;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
  fill_u16_kernel<<<blocks, 256, 0, st>>>(static_cast<unsigned short*>(tau), count,
                                          __bfloat16_as_ushort(__float2bfloat16_rn(v)));
  return check_launch("fill_u16_kernel");
}

int launch_fill(float* a, int n, int ld, float v, cudaStream_t st) {
  const size_t count = (size_t)n * ld;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
  fill_kernel<<<blocks, 256, 0, st>>>(a, count, v);
  return check_launch("fill_kernel");
}

int launch_build_P(const void* tau, int tau_prec, const float* H, int n, int ld, int alpha, float inv_gamma,
                   const float* inv_gamma_dev, const uint32_t* it_dev, int n_sched, int prec,
                   void* P, cudaStream_t st) {
  const bool tb = tau_prec == ACO_BF16;
#define ACO_BUILD_P(PR)                                                                                  \
  do {                                                                                                   \
    if (tb)                                                                                              \
      build_P_kernel<PR, true><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev, it_dev, \
                                                  n_sched, P);                                           \
    else                                                                                                 \
      build_P_kernel<PR, false><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev,       \
                                                   it_dev, n_sched, P);                                  \
  } while (0)
  switch (prec) {
    case ACO_FP32:
      ACO_BUILD_P(ACO_FP32);
      break;
    case ACO_BF16:
      ACO_BUILD_P(ACO_BF16);
      break;
    case ACO_FP16:
      ACO_BUILD_P(ACO_FP16);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
#undef ACO_BUILD_P
  return check_launch("build_P_kernel");
}

int launch_build_P_lists(const void* tau, int tau_prec, const float* H, int n, int ld, int alpha, float inv_gamma,
                         const float* inv_gamma_dev, const uint32_t* it_dev, int n_sched, float rho, int prec, void* P,
                         uint2* lists, int* lcnt, uint32_t* lkey, cudaStream_t st) {
  const bool tb = tau_prec == ACO_BF16;
  const float keep = 1.0f - rho;
#define ACO_BUILD_PL(PR)                                                                                            \
  do {                                                                                                              \
    if (tb)                                                                                                         \
      build_P_lists_kernel<PR, true><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev, it_dev,     \
                                                        n_sched, keep, P, lists, lcnt, lkey);                       \
    else                                                                                                            \
      build_P_lists_kernel<PR, false><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev, it_dev,    \
                                                         n_sched, keep, P, lists, lcnt, lkey);                      \
  } while (0)
  switch (prec) {
    case ACO_FP32:
      ACO_BUILD_PL(ACO_FP32);
      break;
    case ACO_BF16:
      ACO_BUILD_PL(ACO_BF16);
      break;
    case ACO_FP16:
      ACO_BUILD_PL(ACO_FP16);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
#undef ACO_BUILD_PL
  return check_launch("build_P_lists_kernel");
}

int launch_build_lists(const void* P, int prec, int n, int ld, uint2* lists, int* lcnt,
                       uint32_t* lkey, cudaStream_t st) {
  switch (prec) {
    case ACO_FP32:
      build_lists_kernel<ACO_FP32><<<n, 256, 0, st>>>(P, n, ld, lists, lcnt, lkey);
      break;
    case ACO_BF16:
      build_lists_kernel<ACO_BF16><<<n, 256, 0, st>>>(P, n, ld, lists, lcnt, lkey);
      break;
    case ACO_FP16:
      build_lists_kernel<ACO_FP16><<<n, 256, 0, st>>>(P, n, ld, lists, lcnt, lkey);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  return check_launch("build_lists_kernel");
}

// Warps per ant: enough that every warp has a few rounds of four edges per
// lane, and that a thousand ants fill the GPU several times over.
int tour_length_warps(int n) { return n >= 2048 ? 4 : (n >= 512 ? 2 : 1); }

// The paired form: 8 warps per ant (4 of its 512-thread CTAs per SM, one
// wave for m = 1024); staging of 8 bytes per city, at most 56 KB.
constexpr int kTourPairW = 8;
constexpr int kTourPairMaxN = 7168;

int prepare_tour_length() {
  ACO_CUDA_TRY(cudaFuncSetAttribute(tour_length_pair_kernel<kTourPairW, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kTourPairMaxN * 8));
  ACO_CUDA_TRY(cudaFuncSetAttribute(tour_length_pair_kernel<kTourPairW, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kTourPairMaxN * 8));
  return ACO_OK;
}

int launch_tour_length(const double* D, int n, const int32_t* tours, int m, float Q, double* L,
                       double* c, int32_t* nbr, bool packed, cudaStream_t st) {
  const int W = tour_length_warps(n);
#define ACO_TOUR_LENGTH(PK)                                                                                        \
  do {                                                                                                             \
    /* pairs write 16-byte halves of nbr's rows: m even keeps every row aligned */                                \
    if (nbr && W == 4 && n <= kTourPairMaxN && m % 2 == 0 && aligned16(nbr)) {                                     \
      tour_length_pair_kernel<kTourPairW, PK><<<m / 2, 64 * kTourPairW, (size_t)n * 8, st>>>(D, n, tours, m, Q, L, \
                                                                                             c, nbr);              \
      return check_launch("tour_length_pair_kernel");                                                              \
    }                                                                                                              \
    switch (W) {                                                                                                   \
      case 4:                                                                                                      \
        tour_length_kernel<4, PK><<<m, 128, 0, st>>>(D, n, tours, m, Q, L, c, nbr);                                \
        break;                                                                                                     \
      case 2:                                                                                                      \
        tour_length_kernel<2, PK><<<m, 64, 0, st>>>(D, n, tours, m, Q, L, c, nbr);                                 \
        break;                                                                                                     \
      default:                                                                                                     \
        tour_length_kernel<1, PK><<<(m + 7) / 8, 256, 0, st>>>(D, n, tours, m, Q, L, c, nbr);                      \
    }                                                                                                              \
  } while (0)
  if (packed)
    ACO_TOUR_LENGTH(true);
  else
    ACO_TOUR_LENGTH(false);
#undef ACO_TOUR_LENGTH
  return check_launch("tour_length_kernel");
}

int launch_best(const double* L, const int32_t* tours, int n, int m, int32_t* best_tour,
                double* best_len, uint32_t* it_dev, double* c, int topk, int2* dep, int32_t* err,
                cudaStream_t st) {
  best_kernel<<<1, 1024, 0, st>>>(L, tours, n, m, best_tour, best_len, it_dev, c, topk, dep, err);
  return check_launch("best_kernel");
}

int launch_select_topk(const double* L, int m, int k, double* c, cudaStream_t st) {
  select_topk_kernel<<<1, 1024, 0, st>>>(L, m, k, c);
  return check_launch("select_topk_kernel");
}

// The fused kernel's dynamic shared memory: the deposit's, at least the list
// scratch that reuses it.
static size_t deposit_P_smem_bytes(int n, int cap) {
  return std::max(deposit_smem_bytes(n, cap), (size_t)kListScratchWords * 4);
}

int prepare_deposit() {
  const int most = (int)deposit_P_smem_bytes(ACO_MAX_N, kDepCap);
  ACO_CUDA_TRY(cudaFuncSetAttribute(deposit_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
  ACO_CUDA_TRY(cudaFuncSetAttribute(deposit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
  const void* fused[] = {(const void*)deposit_P_lists_kernel<ACO_FP32, false>,
                         (const void*)deposit_P_lists_kernel<ACO_FP32, true>,
                         (const void*)deposit_P_lists_kernel<ACO_BF16, false>,
                         (const void*)deposit_P_lists_kernel<ACO_BF16, true>,
                         (const void*)deposit_P_lists_kernel<ACO_FP16, false>,
                         (const void*)deposit_P_lists_kernel<ACO_FP16, true>};
  for (const void* f : fused)
    ACO_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
  return ACO_OK;
}

int launch_deposit_P_lists(void* tau, int tau_prec, int n, int ld, const int32_t* nbr, const double* c, int m,
                           float rho, const int2* dep, const float* H, int alpha, const float* inv_gamma_dev,
                           const uint32_t* it_dev, int n_sched, int prec, void* P, uint2* lists, int* lcnt,
                           uint32_t* lkey, cudaStream_t st) {
  const int cap = deposit_cap(n, m);
  const size_t smem = deposit_P_smem_bytes(n, cap);
  const float keep = 1.0f - rho;
  const bool tb = tau_prec == ACO_BF16;
#define ACO_DEP_P(PR)                                                                                              \
  do {                                                                                                             \
    if (tb)                                                                                                        \
      deposit_P_lists_kernel<PR, true><<<n, kDepThreads, smem, st>>>(tau, n, ld, nbr, c, m, keep, dep, cap, H,     \
                                                                     alpha, inv_gamma_dev, it_dev, n_sched, P,    \
                                                                     lists, lcnt, lkey);                          \
    else                                                                                                           \
      deposit_P_lists_kernel<PR, false><<<n, kDepThreads, smem, st>>>(tau, n, ld, nbr, c, m, keep, dep, cap, H,    \
                                                                      alpha, inv_gamma_dev, it_dev, n_sched, P,   \
                                                                      lists, lcnt, lkey);                         \
  } while (0)
  switch (prec) {
    case ACO_FP32:
      ACO_DEP_P(ACO_FP32);
      break;
    case ACO_BF16:
      ACO_DEP_P(ACO_BF16);
      break;
    case ACO_FP16:
      ACO_DEP_P(ACO_FP16);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
#undef ACO_DEP_P
  return check_launch("deposit_P_lists_kernel");
}

int launch_deposit(void* tau, int tau_prec, int n, int ld, const int32_t* nbr, const double* c, int m,
                   float rho, const int2* dep, int32_t* err, cudaStream_t st) {
  const int cap = deposit_cap(n, m);
  const size_t smem = deposit_smem_bytes(n, cap);
  const float keep = 1.0f - rho;
  if (tau_prec == ACO_BF16)
    deposit_kernel<true><<<n, kDepThreads, smem, st>>>(tau, n, ld, nbr, c, m, keep, dep, cap, err);
  else
    deposit_kernel<false><<<n, kDepThreads, smem, st>>>(tau, n, ld, nbr, c, m, keep, dep, cap, err);
  return check_launch("deposit_kernel");
}

int launch_deposit_atomic(float* tau, int n, int ld, const int32_t* tours, const double* c, int m,
                          float rho, cudaStream_t st) {
  const float keep = 1.0f - rho;
  dim3 g1((n + 255) / 256, n);
  evaporate_kernel<<<g1, 256, 0, st>>>(tau, n, ld, keep);
  int rc = check_launch("evaporate_kernel");
  if (rc) return rc;
  const size_t total = (size_t)m * n;
  deposit_atomic_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(tau, n, ld, tours, c, m);
  return check_launch("deposit_atomic_kernel");
}

int launch_philox(const uint32_t* ctr, uint2 key, uint32_t* out, int count, cudaStream_t st) {
  philox_kernel<<<(count + 255) / 256, 256, 0, st>>>(ctr, key, out, count);
  return check_launch("philox_kernel");
}

int launch_pow_own(const float* x, float e, float* out, int count, cudaStream_t st) {
  pow_own_kernel<<<(count + 255) / 256, 256, 0, st>>>(x, e, out, count);
  return check_launch("pow_own_kernel");
}

}  // namespace aco
