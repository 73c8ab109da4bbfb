// The non-construction kernels of one TensorACO iteration (sm_103a):
//   heuristic   Sec. 2.1: fp64 distances and eta^beta           (once per instance)
//   build_P     Eq. 1:   M_p = tau^alpha * eta^beta [^(1/gamma)] (per iteration)
//   tour_length Eq. 3:   f(s) in fp64, Q/f, and the index mapping of Eq. 2
//   best        iteration best merged into the running best
//   deposit     Sec. 2.3: evaporation + Delta M_tau (deterministic / atomic)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace aco {

// ---------------------------------------------------------------------------
// Sec. 2.1: D_ij = sqrt(dx^2 + dy^2) (fp64), H_ij = fl32((1/max(d,1e-9))^beta).
// Grid: (ceil(ld/256), n); each thread one (i, j); coalesced row writes.
// ---------------------------------------------------------------------------
__global__ void heuristic_kernel(const float* __restrict__ xy, int n, int beta,
                                 double* __restrict__ D, float* __restrict__ H, int ld) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ld) return;
  if (j >= n) {
    H[(size_t)i * ld + j] = 0.0f;
    return;
  }
  const double dx = __dsub_rn((double)xy[2 * i], (double)xy[2 * j]);
  const double dy = __dsub_rn((double)xy[2 * i + 1], (double)xy[2 * j + 1]);
  const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  if (D) D[(size_t)i * n + j] = d;
  float h = 0.0f;
  if (i != j) h = __double2float_rn(powi_f64(__ddiv_rn(1.0, d > 1e-9 ? d : 1e-9), beta));
  H[(size_t)i * ld + j] = h;
}

__global__ void fill_kernel(float* __restrict__ a, size_t count, float v) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (size_t)gridDim.x * blockDim.x)
    a[q] = v;
}

// ---------------------------------------------------------------------------
// Eq. 1 without row normalisation, one CTA per row, 4 columns per thread step
// (16-byte loads of tau and H).  FP16 rows are scaled by 2^-e_i first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float p_entry(float tau, float h, int i, int j, int n, int alpha,
                                         float inv_gamma) {
  if (j >= n || j == i) return 0.0f;
  float x = __fmul_rn(powi_f32(tau, alpha), h);
  if (inv_gamma != 1.0f) x = pow_own(x, inv_gamma);
  return x;
}

template <int PREC>
__global__ void __launch_bounds__(256) build_P_kernel(const float* __restrict__ tau,
                                                      const float* __restrict__ H, int n, int ld,
                                                      int alpha, float inv_gamma_arg,
                                                      const float* __restrict__ inv_gamma_dev,
                                                      const uint32_t* __restrict__ it_dev,
                                                      int n_sched, void* __restrict__ Pv) {
  const int i = blockIdx.x;
  float inv_gamma = inv_gamma_arg;
  if (inv_gamma_dev) {
    uint32_t it = *it_dev;
    inv_gamma = inv_gamma_dev[it < (uint32_t)n_sched ? it : (uint32_t)(n_sched - 1)];
  }
  const float4* t4 = reinterpret_cast<const float4*>(tau + (size_t)i * ld);
  const float4* h4 = reinterpret_cast<const float4*>(H + (size_t)i * ld);
  const int nq = ld >> 2;

  float scale = 1.0f;
  if (PREC == ACO_FP16) {
    float mx = 0.0f;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const float4 a = __ldg(t4 + q), b = __ldg(h4 + q);
      const int j = 4 * q;
      mx = fmaxf(mx, p_entry(a.x, b.x, i, j, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.y, b.y, i, j + 1, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.z, b.z, i, j + 2, n, alpha, inv_gamma));
      mx = fmaxf(mx, p_entry(a.w, b.w, i, j + 3, n, alpha, inv_gamma));
    }
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(ACO_FULL_MASK, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    int e = 0;
    if (mx > 0.0f) {
      const int ef = (int)((__float_as_uint(mx) >> 23) & 0xFF);
      e = (ef == 0 ? -127 : ef - 127) - 14;
      e = e < -126 ? -126 : (e > 113 ? 113 : e);
    }
    scale = __uint_as_float((uint32_t)(127 - e) << 23);
  }

  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const float4 a = __ldg(t4 + q), b = __ldg(h4 + q);
    const int j = 4 * q;
    const float x0 = p_entry(a.x, b.x, i, j, n, alpha, inv_gamma);
    const float x1 = p_entry(a.y, b.y, i, j + 1, n, alpha, inv_gamma);
    const float x2 = p_entry(a.z, b.z, i, j + 2, n, alpha, inv_gamma);
    const float x3 = p_entry(a.w, b.w, i, j + 3, n, alpha, inv_gamma);
    if (PREC == ACO_FP32) {
      reinterpret_cast<float4*>(Pv)[(size_t)i * nq + q] = make_float4(x0, x1, x2, x3);
    } else if (PREC == ACO_BF16) {
      const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x0)) |
                          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x1)) << 16);
      const uint32_t hi = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x2)) |
                          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x3)) << 16);
      reinterpret_cast<uint2*>(Pv)[(size_t)i * nq + q] = make_uint2(lo, hi);
    } else {
      const uint32_t lo = (uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x0, scale))) |
                          ((uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x1, scale))) << 16);
      const uint32_t hi = (uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x2, scale))) |
                          ((uint32_t)__half_as_ushort(__float2half_rn(__fmul_rn(x3, scale))) << 16);
      reinterpret_cast<uint2*>(Pv)[(size_t)i * nq + q] = make_uint2(lo, hi);
    }
  }
}

// ---------------------------------------------------------------------------
// Eq. 3 + Eq. 2.  One warp per ant: lanes gather 32 consecutive edge lengths
// D[p_t][p_{t+1}] at a time; the fp64 sum is then taken in t order through
// shuffles (the same order as a sequential loop).  The same pass writes the
// index mapping: for city a = p_t, nbr[a][k] = (p_{t-1}, p_{t+1}).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tour_length_kernel(const double* __restrict__ D, int n,
                                                          const int32_t* __restrict__ tours,
                                                          int m, float Q, double* __restrict__ L,
                                                          double* __restrict__ c,
                                                          int32_t* __restrict__ nbr) {
  constexpr int U = 4;  // edge batches of 32 gathered before their sums
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= m) return;
  const int32_t* p = tours + (size_t)k * n;
  double s = 0.0;
  for (int base = 0; base < n; base += 32 * U) {
    double d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * 32 + lane;
      d[u] = 0.0;
      if (t < n) {
        const int a = p[t];
        const int b = p[t + 1 < n ? t + 1 : 0];
        const int pr = p[t > 0 ? t - 1 : n - 1];
        // tours come from the construction kernel; an entry out of range (only
        // after a failed construction, which the host reports) is skipped
        if ((unsigned)a < (unsigned)n && (unsigned)b < (unsigned)n) {
          d[u] = __ldg(D + (size_t)a * n + b);
          if (nbr) reinterpret_cast<int2*>(nbr)[(size_t)a * m + k] = make_int2(pr, b);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int cnt = min(32, n - (base + u * 32));
      for (int q = 0; q < cnt; ++q) s = __dadd_rn(s, __shfl_sync(ACO_FULL_MASK, d[u], q));
    }
  }
  if (lane == 0) {
    L[k] = s;
    if (c) c[k] = __ddiv_rn((double)Q, s);
  }
}

// ---------------------------------------------------------------------------
// Iteration best (lowest ant index on ties) merged into the running best
// (strictly shorter only).  One CTA of 1024 threads.  Also advances the device
// iteration counter, after every kernel of the iteration that reads it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) best_kernel(const double* __restrict__ L,
                                                    const int32_t* __restrict__ tours, int n,
                                                    int m, int32_t* __restrict__ best_tour,
                                                    double* __restrict__ best_len,
                                                    uint32_t* __restrict__ it_dev) {
  __shared__ double sl[32];
  __shared__ int sk[32];
  __shared__ int take;
  double bl = INFINITY;
  int bk = 0x7FFFFFFF;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double v = L[k];
    if (v < bl || (v == bl && k < bk)) {
      bl = v;
      bk = k;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(ACO_FULL_MASK, bl, off);
    const int ok = __shfl_xor_sync(ACO_FULL_MASK, bk, off);
    if (ov < bl || (ov == bl && ok < bk)) {
      bl = ov;
      bk = ok;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sl[threadIdx.x >> 5] = bl;
    sk[threadIdx.x >> 5] = bk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (sl[w] < bl || (sl[w] == bl && sk[w] < bk)) {
        bl = sl[w];
        bk = sk[w];
      }
    }
    take = (bk < m && bl < *best_len) ? 1 : 0;
    sk[0] = bk;
    if (take) *best_len = bl;
    if (it_dev) *it_dev = *it_dev + 1u;
  }
  __syncthreads();
  if (take) {
    const int32_t* src = tours + (size_t)sk[0] * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) best_tour[t] = src[t];
  }
}

// ---------------------------------------------------------------------------
// Sec. 2.3 deterministic deposit.  One warp per row a of tau.  The row's
// pheromone increment Delta_a. is accumulated in fp64 shared memory; the
// 2m index-mapping entries of the row (two neighbours per ant) are taken 16
// ants at a time: lanes 0-15 hold the predecessors, lanes 16-31 the
// successors.  __match_any_sync groups lanes with the same target column b;
// the lane of the lowest ant in a group adds the group's c_k to Delta_ab in
// ascending k, so every Delta_ab is summed in ascending ant order.  Columns
// are processed in tiles of `tile` (shared memory), ants in chunks of 1024.
// ---------------------------------------------------------------------------
constexpr int kDepAntChunk = 1024;

__global__ void __launch_bounds__(32) deposit_kernel(float* __restrict__ tau, int n, int ld,
                                                     const int32_t* __restrict__ nbr,
                                                     const double* __restrict__ c, int m,
                                                     double keep, int tile) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* delta = reinterpret_cast<double*>(smem);              // [tile]
  double* cs = delta + tile;                                    // [kDepAntChunk]
  int2* items = reinterpret_cast<int2*>(cs + kDepAntChunk);     // [kDepAntChunk]
  const int a = blockIdx.x;
  const int lane = threadIdx.x;
  float* row = tau + (size_t)a * ld;

  for (int col0 = 0; col0 < n; col0 += tile) {
    const int cols = min(tile, n - col0);
    for (int q = lane; q < cols; q += 32) delta[q] = 0.0;
    for (int kb = 0; kb < m; kb += kDepAntChunk) {
      const int cnt = min(kDepAntChunk, m - kb);
      __syncwarp();
      const int2* src = reinterpret_cast<const int2*>(nbr) + ((size_t)a * m + kb);
#pragma unroll 4
      for (int q = lane; q < cnt; q += 32) {
        items[q] = __ldg(src + q);
        cs[q] = __ldg(c + kb + q);
      }
      __syncwarp();
      for (int k0 = 0; k0 < cnt; k0 += 16) {
        const int ai = lane & 15;  // ant k0 + ai
        const bool valid = k0 + ai < cnt;
        int b = -1;
        if (valid) {
          const int2 it = items[k0 + ai];
          b = (lane >> 4 ? it.y : it.x) - col0;
        }
        const bool in_tile = valid && b >= 0 && b < cols;
        const int key = in_tile ? b : -1 - lane;  // unique keys for idle lanes
        const unsigned grp = __match_any_sync(ACO_FULL_MASK, key);
        if (in_tile) {
          const unsigned ants = (grp & 0xFFFFu) | (grp >> 16);
          const int lead = __ffs(ants) - 1;
          if (lead == ai) {
            double sum = delta[b];
            unsigned rest = ants;
            while (rest) {
              const int i = __ffs(rest) - 1;
              rest &= rest - 1u;
              sum = __dadd_rn(sum, cs[k0 + i]);
            }
            delta[b] = sum;
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();
    // tau_ab <- fl32(fl64(keep * tau_ab) + Delta_ab), four columns per lane step
    const int nv = cols >> 2;
    float4* row4 = reinterpret_cast<float4*>(row + col0);
#pragma unroll 4
    for (int q = lane; q < nv; q += 32) {
      float4 v = row4[q];
      const double* dl = delta + 4 * q;
      v.x = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.x), dl[0]));
      v.y = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.y), dl[1]));
      v.z = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.z), dl[2]));
      v.w = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)v.w), dl[3]));
      row4[q] = v;
    }
    for (int q = 4 * nv + lane; q < cols; q += 32) {
      const int j = col0 + q;
      row[j] = __double2float_rn(__dadd_rn(__dmul_rn(keep, (double)row[j]), delta[q]));
    }
  }
}

__global__ void evaporate_kernel(float* __restrict__ tau, int n, int ld, double keep) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float* p = tau + (size_t)i * ld + j;
  *p = __double2float_rn(__dmul_rn(keep, (double)*p));
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

// ------------------------------------------------------------------ launchers
static int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ACO_OK : cuda_error(e, what);
}

int launch_heuristic(const float* xy, int n, int beta, double* D, float* H, int ld,
                     cudaStream_t st) {
  dim3 grid((ld + 255) / 256, n);
  heuristic_kernel<<<grid, 256, 0, st>>>(xy, n, beta, D, H, ld);
  return check_launch("heuristic_kernel");
}

int launch_fill(float* a, int n, int ld, float v, cudaStream_t st) {
  const size_t count = (size_t)n * ld;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
  fill_kernel<<<blocks, 256, 0, st>>>(a, count, v);
  return check_launch("fill_kernel");
}

int launch_build_P(const float* tau, const float* H, int n, int ld, int alpha, float inv_gamma,
                   const float* inv_gamma_dev, const uint32_t* it_dev, int n_sched, int prec,
                   void* P, cudaStream_t st) {
  switch (prec) {
    case ACO_FP32:
      build_P_kernel<ACO_FP32><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev,
                                                 it_dev, n_sched, P);
      break;
    case ACO_BF16:
      build_P_kernel<ACO_BF16><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev,
                                                 it_dev, n_sched, P);
      break;
    case ACO_FP16:
      build_P_kernel<ACO_FP16><<<n, 256, 0, st>>>(tau, H, n, ld, alpha, inv_gamma, inv_gamma_dev,
                                                 it_dev, n_sched, P);
      break;
    default:
      return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  }
  return check_launch("build_P_kernel");
}

int launch_tour_length(const double* D, int n, const int32_t* tours, int m, float Q, double* L,
                       double* c, int32_t* nbr, cudaStream_t st) {
  tour_length_kernel<<<(m + 7) / 8, 256, 0, st>>>(D, n, tours, m, Q, L, c, nbr);
  return check_launch("tour_length_kernel");
}

int launch_best(const double* L, const int32_t* tours, int n, int m, int32_t* best_tour,
                double* best_len, uint32_t* it_dev, cudaStream_t st) {
  best_kernel<<<1, 1024, 0, st>>>(L, tours, n, m, best_tour, best_len, it_dev);
  return check_launch("best_kernel");
}

int deposit_tile(int n) {
  // fp64 delta tile + per-chunk c and items must fit the 227 KB opt-in limit
  // (a multiple of 4 so that every tile's columns start 16-byte aligned)
  const int max_tile = ((200 * 1024 - kDepAntChunk * 16) / 8) & ~3;
  return n < max_tile ? n : max_tile;
}

int prepare_deposit() {
  ACO_CUDA_TRY(cudaFuncSetAttribute(deposit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
  return ACO_OK;
}

int launch_deposit(float* tau, int n, int ld, const int32_t* nbr, const double* c, int m,
                   float rho, cudaStream_t st) {
  const int tile = deposit_tile(n);
  const size_t smem = (size_t)tile * 8 + (size_t)kDepAntChunk * 16;
  const double keep = 1.0 - (double)rho;
  deposit_kernel<<<n, 32, smem, st>>>(tau, n, ld, nbr, c, m, keep, tile);
  return check_launch("deposit_kernel");
}

int launch_deposit_atomic(float* tau, int n, int ld, const int32_t* tours, const double* c, int m,
                          float rho, cudaStream_t st) {
  const double keep = 1.0 - (double)rho;
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
