// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tensoraco.h"

namespace aco {

int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
// status for a nonzero kernel error word: ACO_ERR_TIMEOUT for a wait that
// ran out (kErrTimeout), ACO_ERR_CUDA for any other kernel-side check
int kernel_check_error(int32_t code);

#define ACO_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return ::aco::cuda_error(_e, #expr); \
  } while (0)

#define ACO_CHECK_LAUNCH(what)                              \
  do {                                                      \
    cudaError_t _e = cudaGetLastError();                    \
    if (_e != cudaSuccess) return ::aco::cuda_error(_e, what); \
  } while (0)

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Construct-kernel launch shapes compiled in, per element size (4 or 2 bytes).
struct ConstructShape {
  int warps;   // warps per ant
  int chunks;  // 16-byte chunks per lane
  int mode;    // 0: row staged in shared memory by cp.async, 1: direct register loads
};
int construct_shapes(int elem_bytes, const ConstructShape** list);
// Default shape for (n, m, elem_bytes) unless an autotuned choice is registered:
// a direct-load shape with the fewest warps, then fewest chunks, that covers n;
// a staged shape only when no direct shape covers n.
ConstructShape default_construct_shape(int n, int m, int elem_bytes);
void register_tuned_shape(int n, int m, int elem_bytes, ConstructShape s);

// Kernel launchers (return ACO_OK or an error code; asynchronous).
// lists/lcnt/lkey: the candidate lists of M_p (nullptr: full scan only)
int launch_construct_f32(const float* P, int n, int ld, int m, uint2 key, uint32_t it,
                         const uint32_t* it_dev, int32_t* tours, int32_t* err, int warps,
                         int chunks, int mode, const uint2* lists, const int* lcnt,
                         const uint32_t* lkey, cudaStream_t st);
int launch_construct_bf16(const void* P, int n, int ld, int m, uint2 key, uint32_t it,
                          const uint32_t* it_dev, int32_t* tours, int32_t* err, int warps,
                          int chunks, int mode, const uint2* lists, const int* lcnt,
                          const uint32_t* lkey, cudaStream_t st);
int launch_construct_f16(const void* P, int n, int ld, int m, uint2 key, uint32_t it,
                         const uint32_t* it_dev, int32_t* tours, int32_t* err, int warps,
                         int chunks, int mode, const uint2* lists, const int* lcnt,
                         const uint32_t* lkey, cudaStream_t st);
int launch_build_lists(const void* P, int prec, int n, int ld, uint2* lists, int* lcnt,
                       uint32_t* lkey, cudaStream_t st);

struct InstDev;
// bitmap_bytes: shared bytes of the list phase's visited bitmap (0: no lists)
int launch_batch_construct_f32(const InstDev* insts, const int* ant_off, int count, int total,
                               int* counter, int32_t* err, int warps, int chunks, int mode,
                               int bitmap_bytes, int num_sms, cudaStream_t st);
int launch_batch_construct_bf16(const InstDev* insts, const int* ant_off, int count, int total,
                                int* counter, int32_t* err, int warps, int chunks, int mode,
                                int bitmap_bytes, int num_sms, cudaStream_t st);
int launch_batch_construct_f16(const InstDev* insts, const int* ant_off, int count, int total,
                               int* counter, int32_t* err, int warps, int chunks, int mode,
                               int bitmap_bytes, int num_sms, cudaStream_t st);
int batch_construct_shapes(int elem_bytes, const ConstructShape** list);

// Lean (candidate-list) construction, any n <= 16384, one warp per ant
// (mode 2 of a ConstructShape; lists may be null: compact full scans only).
int launch_construct_lean(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                          const uint32_t* it_dev, int32_t* tours, int32_t* err, const uint2* lists,
                          const int* lcnt, const uint32_t* lkey, cudaStream_t st);
int launch_batch_construct_lean(const InstDev* insts, const int* ant_off, int count, int total,
                                int* counter, int32_t* err, int prec, int min_n, int max_n, int num_sms,
                                cudaStream_t st);
int prepare_construct_lean();
// Roulette-wheel construction (Sec. 2.4 baseline), n <= 16384, one 256-thread CTA per ant.
// polls: bound on each step's wait for its row copy (kRwWaitPolls by default);
// a wait that runs out sets *err to kErrTimeout.
constexpr uint32_t kRwWaitPolls = ACO_WAIT_POLLS_DEFAULT;
int launch_construct_rw(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                        const uint32_t* it_dev, int32_t* tours, int32_t* err, uint32_t polls, cudaStream_t st);
// Every ant of `count` roulette-wheel instances (insts; ant_off: exclusive
// prefix sums of their ant counts, `total` ants; max_n: their largest n).
int launch_batch_construct_rw(const InstDev* insts, const int* ant_off, int count, int total, int32_t* err,
                              int prec, int max_n, cudaStream_t st);
int prepare_construct_rw();
constexpr int kModeLean = 2;
constexpr int kLeanMaxN = 16384;
constexpr int kRwMaxN = ACO_MAX_N_RW;

int prepare_construct_f32();
int prepare_construct_bf16();
int prepare_construct_f16();
int prepare_deposit();
int prepare_kernels();  // once per process: shared-memory opt-ins (not during capture)

// packed: D is the strictly upper triangle (tri_index; the solvers' and
// batches' own layout), else n x n (the step-level calls' layout)
int launch_heuristic(const float* xy, int n, int beta, double* D, float* H, int ld, bool packed,
                     cudaStream_t st);
int launch_fill(float* a, int n, int ld, float v, cudaStream_t st);
// tau stored in fp32 (tau_prec ACO_FP32) or bfloat16 (ACO_BF16), leading dimension ld
int launch_build_P(const void* tau, int tau_prec, const float* H, int n, int ld, int alpha, float inv_gamma,
                   const float* inv_gamma_dev, const uint32_t* it_dev, int n_sched, int prec,
                   void* P, cudaStream_t st);
int launch_fill_tau(void* tau, int tau_prec, int n, int ld, float v, cudaStream_t st);
// build_P and build_lists in one pass (the list threshold guessed from the
// previous iteration's bound in lkey; same lists as launch_build_lists)
int launch_build_P_lists(const void* tau, int tau_prec, const float* H, int n, int ld, int alpha, float inv_gamma,
                         const float* inv_gamma_dev, const uint32_t* it_dev, int n_sched, float rho, int prec, void* P,
                         uint2* lists, int* lcnt, uint32_t* lkey, cudaStream_t st);
// the deterministic deposit, then the next iteration's M_p and lists, one
// CTA per row (dep from the best kernel; *it_dev already advanced)
int launch_deposit_P_lists(void* tau, int tau_prec, int n, int ld, const int32_t* nbr, const double* c, int m,
                           float rho, const int2* dep, const float* H, int alpha, const float* inv_gamma_dev,
                           const uint32_t* it_dev, int n_sched, int prec, void* P, uint2* lists, int* lcnt,
                           uint32_t* lkey, cudaStream_t st);
int prepare_tour_length();
int launch_tour_length(const double* D, int n, const int32_t* tours, int m, float Q,
                       double* L, double* c, int32_t* nbr, bool packed, cudaStream_t st);
// best also keeps only the topk shortest paths' weights in c (c non-null,
// 0 < topk < m) and derives the deposit weights' scale into *dep (non-null)
int launch_best(const double* L, const int32_t* tours, int n, int m, int32_t* best_tour,
                double* best_len, uint32_t* it_dev, double* c, int topk, int2* dep, int32_t* err,
                cudaStream_t st);
int launch_select_topk(const double* L, int m, int k, double* c, cudaStream_t st);
// dep null: every CTA derives the scaling from c; err (nullable) gets
// kErrDepositRange when the weights cannot be summed exactly
int launch_deposit(void* tau, int tau_prec, int n, int ld, const int32_t* nbr, const double* c, int m,
                   float rho, const int2* dep, int32_t* err, cudaStream_t st);
int launch_deposit_atomic(float* tau, int n, int ld, const int32_t* tours, const double* c,
                          int m, float rho, cudaStream_t st);
int launch_philox(const uint32_t* ctr, uint2 key, uint32_t* out, int count, cudaStream_t st);
int launch_pow_own(const float* x, float e, float* out, int count, cudaStream_t st);

}  // namespace aco
