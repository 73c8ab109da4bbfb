// Batches: many independent TSP instances advanced together.
//
// Every step of an iteration is one launch over all active instances:
//   build_P      one CTA per (instance, row): M_p and its candidate list in one pass
//   construct    one persistent launch; CTAs pull (instance, ant) items from a
//                global counter, biggest instances first
//   tour_length  one warp per (instance, ant)
//   best         one CTA per instance
//   deposit      one warp per (instance, row)
// The launches of one iteration are captured into a CUDA graph and replayed
// while the set of active instances does not change.  Instance workspaces
// (same layout as a single solver) are carved from one device arena by a
// first-fit allocator; an instance is admitted only if its workspace fits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "internal.h"
#include "steps.cuh"

namespace aco {

// ------------------------------------------------------------------ kernels
// M_p and (for instances with lists) the candidate list of one row per CTA,
// in one pass (build_P_lists_row); the list threshold is guessed from the
// row's previous bound as in the single-instance kernel.
template <int PREC>
__global__ void __launch_bounds__(256) batch_build_P_lists_kernel(const InstDev* __restrict__ insts,
                                                                  const int* __restrict__ row_off, int count) {
  __shared__ uint32_t scratch[kListScratchWords];
  __shared__ float red[32];
  const int r = blockIdx.x;
  const int i = find_instance(row_off, count, r);
  const InstDev& I = insts[i];
  const int row = r - __ldg(row_off + i);
  float inv_gamma = 1.0f, ig_prev = 1.0f;
  if (I.adair) {
    const uint32_t it = *I.it;
    const uint32_t last = (uint32_t)(I.n_sched - 1);
    inv_gamma = I.sched[it < last ? it : last];
    ig_prev = it > 0u ? I.sched[it - 1u < last ? it - 1u : last] : 0.0f;
  }
  const size_t eb = PREC == ACO_FP32 ? 4 : 2;
  void* P_row = static_cast<char*>(I.P) + (size_t)row * I.ld * eb;
  const char* tau_row = reinterpret_cast<const char*>(I.tau) + (size_t)row * I.ld * (I.tau_bf16 ? 2 : 4);
  const float* H_row = I.H + (size_t)row * I.ld;
  if (!I.lists) {
    if (I.tau_bf16)
      build_P_row<PREC, true>(tau_row, H_row, I.n, I.ld, row, I.alpha, inv_gamma, P_row, red);
    else
      build_P_row<PREC, false>(tau_row, H_row, I.n, I.ld, row, I.alpha, inv_gamma, P_row, red);
    return;
  }
  const uint32_t guess = list_guess(I.lkey[row], 1.0f - I.rho, I.alpha, inv_gamma, ig_prev);
  uint2* list = I.lists + (size_t)row * kListMax;
  if (I.tau_bf16)
    build_P_lists_row<PREC, true>(tau_row, H_row, I.n, I.ld, row, I.alpha, inv_gamma, P_row, list, I.lcnt + row,
                                  I.lkey + row, guess, scratch, red);
  else
    build_P_lists_row<PREC, false>(tau_row, H_row, I.n, I.ld, row, I.alpha, inv_gamma, P_row, list, I.lcnt + row,
                                   I.lkey + row, guess, scratch, red);
}

__global__ void __launch_bounds__(256) batch_tour_length_kernel(const InstDev* __restrict__ insts,
                                                                const int* __restrict__ ant_off,
                                                                int count, int total) {
  __shared__ unsigned long long sacc[8 * (kLenDigits + 1)];
  const int wid = (int)(threadIdx.x >> 5);
  const int item = blockIdx.x * (blockDim.x >> 5) + wid;
  if (item >= total) return;
  const int i = find_instance(ant_off, count, item);
  const InstDev& I = insts[i];
  const int k = item - __ldg(ant_off + i);
  tour_length_exact<1, false, true>(I.D, I.n, I.tours + (size_t)k * I.n, k, I.Q, I.L, I.c,
                       I.nbr ? static_cast<void*>(reinterpret_cast<int2*>(I.nbr) + k) : nullptr, I.m, 0,
                       sacc + wid * (kLenDigits + 1));
}

__global__ void __launch_bounds__(256) batch_best_kernel(const InstDev* __restrict__ insts,
                                                         int32_t* __restrict__ err) {
  __shared__ double sl[32];
  __shared__ int sk[33];
  __shared__ int sred[300];
  const InstDev& I = insts[blockIdx.x];
  best_block(I.L, I.tours, I.n, I.m, I.best_tour, I.best_len, I.it, sl, sk);
  select_topk_block(I.L, I.m, I.topk, I.c, sred);
  const int2 d = deposit_scale_block(I.c, I.m, sred);
  if (threadIdx.x == 0) {
    *I.dep = d;
    if (d.y == kDepBad && err) atomicExch(err, kErrDepositRange);
  }
}

__global__ void __launch_bounds__(kDepThreads) batch_deposit_kernel(const InstDev* __restrict__ insts,
                                                                    const int* __restrict__ row_off,
                                                                    int count) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = blockIdx.x;
  const int i = find_instance(row_off, count, r);
  const InstDev& I = insts[i];
  const int a = r - __ldg(row_off + i);
  const int2 d = *I.dep;
  const int2* nbr_row = reinterpret_cast<const int2*>(I.nbr) + (size_t)a * I.m;
  char* tau_row = reinterpret_cast<char*>(I.tau) + (size_t)a * I.ld * (I.tau_bf16 ? 2 : 4);
  if (I.tau_bf16)
    deposit_row_exact<true>(tau_row, I.n, nbr_row, I.c, I.m, 1.0f - I.rho, d.x, d.y, deposit_cap(I.n, I.m), smem);
  else
    deposit_row_exact<false>(tau_row, I.n, nbr_row, I.c, I.m, 1.0f - I.rho, d.x, d.y, deposit_cap(I.n, I.m), smem);
}

// ------------------------------------------------------------------ arena
// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    used_.clear();
    if (size) free_[0] = size;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_[*off] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t at = off, bytes = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(at);
    if (next != free_.end() && at + bytes == next->first) {
      bytes += next->second;
      free_.erase(next);
    }
    auto it = free_.lower_bound(at);
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == at) {
        at = prev->first;
        bytes += prev->second;
        free_.erase(prev);
      }
    }
    free_[at] = bytes;
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto& f : free_) s += f.second;
    return s;
  }
  size_t largest() const {
    size_t s = 0;
    for (auto& f : free_) s = std::max(s, f.second);
    return s;
  }

 private:
  std::map<size_t, size_t> free_, used_;
  size_t size_ = 0;
};

struct Slot {
  bool used = false;
  aco_params p{};
  size_t off = 0;
  InstDev dev{};
  uint32_t done = 0;      // iterations completed
  int budget = 0;         // iterations to run (0: unlimited)
  bool finished() const { return budget > 0 && (int)done >= budget; }
};

// Per-instance helpers from solver.cu (workspace layout, schedule values).
size_t instance_workspace_bytes(int n, int m);
int instance_bind(const aco_params& p, unsigned char* ws, InstDev* d, cudaStream_t st,
                  const float* coords_host);

}  // namespace aco

using namespace aco;

struct aco_batch {
  int prec = ACO_FP32;
  cudaStream_t stream = nullptr;
  unsigned char* arena_mem = nullptr;
  bool own_arena = false;
  size_t arena_bytes = 0;
  Arena arena;
  std::vector<Slot> slots;
  int num_sms = 0;
  // device tables of the active set
  InstDev* d_insts = nullptr;
  int* d_row_off = nullptr;
  int* d_ant_off = nullptr;
  int* d_counter = nullptr;
  int32_t* d_err = nullptr;
  std::vector<int> active;      // slot ids, n descending
  InstDev* d_ir_insts = nullptr;  // the IR / AdaIR instances of the active set
  int* d_ir_off = nullptr;        // their ants' exclusive prefix sums
  InstDev* d_rw_insts = nullptr;  // the roulette-wheel instances
  int* d_rw_off = nullptr;
  std::vector<int> ir;            // positions in `active` of the IR / AdaIR instances
  int total_rows = 0, total_ants = 0;
  int min_n = 0, max_n = 0, ir_ants = 0;  // over the IR / AdaIR instances
  int rw_count = 0, rw_ants = 0, rw_max_n = 0;
  size_t dep_smem = 0;          // deposit shared memory of the largest instance
  ConstructShape shape{0, 0, 0};  // forced shape for every class ({0,0,0}: per class)
  struct Class {  // first, count: a range of the IR / AdaIR table
    int first, count, total;
    ConstructShape s;
  };
  std::vector<Class> classes;     // contiguous ranges of `active` sharing a shape
  bool lean = false;              // all IR / AdaIR instances use candidate lists: lean kernel
  bool tables_ok = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace aco {

constexpr int kMaxClasses = 32;

static void batch_drop_graph(aco_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

static int batch_shape_columns(ConstructShape s, int eb) { return 32 * s.warps * s.chunks * (16 / eb); }

static ConstructShape batch_default_shape(int max_n, int eb) {
  const ConstructShape* list;
  const int cnt = batch_construct_shapes(eb, &list);
  ConstructShape best = {0, 0, 0};
  for (int q = 0; q < cnt; ++q) {
    const ConstructShape s = list[q];
    if (batch_shape_columns(s, eb) < max_n) continue;
    const bool better = best.warps == 0 || s.mode > best.mode ||
                        (s.mode == best.mode && (s.warps < best.warps ||
                                                 (s.warps == best.warps && s.chunks < best.chunks)));
    if (better) best = s;
  }
  return best;
}

// Rebuild the active set (unfinished instances, n descending) and its tables.
static int batch_refresh(aco_batch* b) {
  b->active.clear();
  for (int q = 0; q < (int)b->slots.size(); ++q)
    if (b->slots[q].used && !b->slots[q].finished()) b->active.push_back(q);
  std::stable_sort(b->active.begin(), b->active.end(),
                   [&](int x, int y) { return b->slots[x].p.n > b->slots[y].p.n; });
  const int cnt = (int)b->active.size();
  // every instance (build_P, lists, lengths, best, deposit); the IR / AdaIR
  // ones (their construction kernels); the roulette-wheel ones (theirs)
  std::vector<InstDev> insts(cnt), ir_insts, rw_insts;
  std::vector<int> row_off(cnt + 1, 0), ant_off(cnt + 1, 0), ir_off(1, 0), rw_off(1, 0);
  b->ir.clear();
  b->max_n = 0;
  b->min_n = 0;
  b->rw_max_n = 0;
  b->dep_smem = 0;
  for (int q = 0; q < cnt; ++q) {
    const Slot& s = b->slots[b->active[q]];
    insts[q] = s.dev;
    row_off[q + 1] = row_off[q] + s.p.n;
    ant_off[q + 1] = ant_off[q] + s.p.m;
    if (s.dev.rw) {
      rw_insts.push_back(s.dev);
      rw_off.push_back(rw_off.back() + s.p.m);
      b->rw_max_n = std::max(b->rw_max_n, s.p.n);
    } else {
      b->ir.push_back(q);
      ir_insts.push_back(s.dev);
      ir_off.push_back(ir_off.back() + s.p.m);
      b->min_n = b->max_n == 0 ? s.p.n : std::min(b->min_n, s.p.n);
      b->max_n = std::max(b->max_n, s.p.n);
    }
    b->dep_smem = std::max(b->dep_smem, deposit_smem_bytes(s.p.n, deposit_cap(s.p.n, s.p.m)));
  }
  b->total_rows = row_off[cnt];
  b->total_ants = ant_off[cnt];
  b->ir_ants = ir_off.back();
  b->rw_count = (int)rw_insts.size();
  b->rw_ants = rw_off.back();
  const int ir_cnt = (int)b->ir.size();
  auto put = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->stream) : cudaSuccess;
  };
  if (cnt) {
    ACO_CUDA_TRY(put(b->d_insts, insts.data(), sizeof(InstDev) * cnt));
    ACO_CUDA_TRY(put(b->d_row_off, row_off.data(), sizeof(int) * (cnt + 1)));
    ACO_CUDA_TRY(put(b->d_ant_off, ant_off.data(), sizeof(int) * (cnt + 1)));
    ACO_CUDA_TRY(put(b->d_ir_insts, ir_insts.data(), sizeof(InstDev) * ir_cnt));
    ACO_CUDA_TRY(put(b->d_ir_off, ir_off.data(), sizeof(int) * (ir_cnt + 1)));
    ACO_CUDA_TRY(put(b->d_rw_insts, rw_insts.data(), sizeof(InstDev) * b->rw_count));
    ACO_CUDA_TRY(put(b->d_rw_off, rw_off.data(), sizeof(int) * (b->rw_count + 1)));
    ACO_CUDA_TRY(cudaStreamSynchronize(b->stream));  // pageable sources
  }
  // IR / AdaIR instances: the lean kernel when all of them have candidate
  // lists (and no shape is forced); else size classes: consecutive instances
  // (n descending) sharing a shape.  Indices below are into their table.
  const int eb = b->prec == ACO_FP32 ? 4 : 2;
  b->lean = ir_cnt > 0 && b->shape.warps == 0 && b->max_n <= kLeanMaxN;
  for (int q = 0; q < ir_cnt; ++q) b->lean = b->lean && b->slots[b->active[b->ir[q]]].p.cand_lists;
  b->classes.clear();
  for (int q = 0; q < ir_cnt; ++q) {
    const Slot& sl = b->slots[b->active[b->ir[q]]];
    ConstructShape s = b->shape;
    if (s.warps == 0 || batch_shape_columns(s, eb) < sl.p.n) s = batch_default_shape(sl.p.n, eb);
    if (s.warps == 0) return set_error(ACO_ERR_UNSUPPORTED, "no batch construct shape covers n=%d", sl.p.n);
    if (!b->classes.empty()) {
      auto& c = b->classes.back();
      if (c.s.warps == s.warps && c.s.chunks == s.chunks && c.s.mode == s.mode) {
        c.count += 1;
        c.total += sl.p.m;
        continue;
      }
    }
    if ((int)b->classes.size() == kMaxClasses) {  // merge into the last class (its shape covers smaller n)
      b->classes.back().count += 1;
      b->classes.back().total += sl.p.m;
      continue;
    }
    b->classes.push_back({q, 1, sl.p.m, s});
  }
  batch_drop_graph(b);
  b->tables_ok = true;
  return ACO_OK;
}

static int batch_enqueue(aco_batch* b) {
  const int cnt = (int)b->active.size();
  if (!cnt) return ACO_OK;
  cudaStream_t st = b->stream;
  switch (b->prec) {
    case ACO_FP32:
      batch_build_P_lists_kernel<ACO_FP32><<<b->total_rows, 256, 0, st>>>(b->d_insts, b->d_row_off, cnt);
      break;
    case ACO_BF16:
      batch_build_P_lists_kernel<ACO_BF16><<<b->total_rows, 256, 0, st>>>(b->d_insts, b->d_row_off, cnt);
      break;
    default:
      batch_build_P_lists_kernel<ACO_FP16><<<b->total_rows, 256, 0, st>>>(b->d_insts, b->d_row_off, cnt);
  }
  ACO_CHECK_LAUNCH("batch_build_P_lists_kernel");
  ACO_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(int) * std::max<size_t>(1, b->classes.size()), st));
  if (b->rw_count) {  // one CTA per roulette-wheel ant
    const int rc = launch_batch_construct_rw(b->d_rw_insts, b->d_rw_off, b->rw_count, b->rw_ants, b->d_err,
                                             b->prec, b->rw_max_n, st);
    if (rc) return rc;
  }
  const int ir_cnt = (int)b->ir.size();
  if (b->lean) {  // one persistent lean launch over every ant of every IR / AdaIR instance
    const int rc = launch_batch_construct_lean(b->d_ir_insts, b->d_ir_off, ir_cnt, b->ir_ants, b->d_counter,
                                               b->d_err, b->prec, b->min_n, b->max_n, b->num_sms, st);
    if (rc) return rc;
  }
  for (size_t ci = 0; ci < (b->lean ? 0 : b->classes.size()); ++ci) {
    const auto& c = b->classes[ci];
    const ConstructShape s = c.s;
    const InstDev* ins = b->d_ir_insts + c.first;
    const int* off = b->d_ir_off + c.first;
    int* ctr = b->d_counter + ci;
    const int bitmap = ((b->slots[b->active[b->ir[c.first]]].p.n + 127) / 128) * 16;  // largest n of the class
    int rc;
    if (b->prec == ACO_FP32)
      rc = launch_batch_construct_f32(ins, off, c.count, c.total, ctr, b->d_err, s.warps, s.chunks, s.mode,
                                      bitmap, b->num_sms, st);
    else if (b->prec == ACO_BF16)
      rc = launch_batch_construct_bf16(ins, off, c.count, c.total, ctr, b->d_err, s.warps, s.chunks, s.mode,
                                       bitmap, b->num_sms, st);
    else
      rc = launch_batch_construct_f16(ins, off, c.count, c.total, ctr, b->d_err, s.warps, s.chunks, s.mode,
                                      bitmap, b->num_sms, st);
    if (rc) return rc;
  }
  batch_tour_length_kernel<<<(b->total_ants + 7) / 8, 256, 0, st>>>(b->d_insts, b->d_ant_off, cnt,
                                                                    b->total_ants);
  ACO_CHECK_LAUNCH("batch_tour_length_kernel");
  batch_best_kernel<<<cnt, 256, 0, st>>>(b->d_insts, b->d_err);
  ACO_CHECK_LAUNCH("batch_best_kernel");
  batch_deposit_kernel<<<b->total_rows, kDepThreads, b->dep_smem, st>>>(b->d_insts, b->d_row_off, cnt);
  ACO_CHECK_LAUNCH("batch_deposit_kernel");
  return ACO_OK;
}

static int batch_capture(aco_batch* b) {
  batch_drop_graph(b);
  ACO_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = batch_enqueue(b);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture(batch)");
  const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
  if (e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_error(e2, "cudaGraphInstantiate(batch)");
  }
  b->graph = g;
  return ACO_OK;
}

}  // namespace aco

extern "C" {

int aco_batch_create(aco_batch** out, int max_instances, size_t arena_bytes, int prec,
                     void* dev_arena, void* stream) {
  if (!out) return set_error(ACO_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (max_instances < 1 || max_instances > (1 << 20)) return set_error(ACO_ERR_ARG, "max_instances out of range");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  if (arena_bytes < 256) return set_error(ACO_ERR_ARG, "arena too small");
  if (dev_arena && ((uintptr_t)dev_arena & 255u)) return set_error(ACO_ERR_ARG, "arena must be 256-byte aligned");
  int rc = prepare_kernels();
  if (rc) return rc;
  // the deposit's slot table may exceed the default 48 KB of dynamic shared memory
  ACO_CUDA_TRY(cudaFuncSetAttribute(batch_deposit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)deposit_smem_bytes(ACO_MAX_N, kDepCap)));
  aco_batch* b = new aco_batch();
  b->prec = prec;
  b->stream = static_cast<cudaStream_t>(stream);
  b->slots.resize(max_instances);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  auto fail = [&](int code) {
    if (b->own_arena && b->arena_mem) cudaFree(b->arena_mem);
    cudaFree(b->d_insts);
    cudaFree(b->d_row_off);
    cudaFree(b->d_ant_off);
    cudaFree(b->d_ir_insts);
    cudaFree(b->d_ir_off);
    cudaFree(b->d_rw_insts);
    cudaFree(b->d_rw_off);
    cudaFree(b->d_counter);
    cudaFree(b->d_err);
    delete b;
    return code;
  };
  if (dev_arena) {
    b->arena_mem = static_cast<unsigned char*>(dev_arena);
  } else {
    const cudaError_t e = cudaMalloc(&b->arena_mem, arena_bytes);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc(batch arena)"));
    b->own_arena = true;
  }
  b->arena_bytes = arena_bytes;
  b->arena.reset(arena_bytes);
  if (cudaMalloc(&b->d_insts, sizeof(InstDev) * max_instances) != cudaSuccess ||
      cudaMalloc(&b->d_row_off, sizeof(int) * (max_instances + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_ant_off, sizeof(int) * (max_instances + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_ir_insts, sizeof(InstDev) * max_instances) != cudaSuccess ||
      cudaMalloc(&b->d_ir_off, sizeof(int) * (max_instances + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_rw_insts, sizeof(InstDev) * max_instances) != cudaSuccess ||
      cudaMalloc(&b->d_rw_off, sizeof(int) * (max_instances + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(int) * kMaxClasses) != cudaSuccess ||
      cudaMalloc(&b->d_err, sizeof(int32_t)) != cudaSuccess)
    return fail(cuda_error(cudaGetLastError(), "cudaMalloc(batch tables)"));
  if (cudaMemset(b->d_err, 0, sizeof(int32_t)) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "memset"));
  *out = b;
  return ACO_OK;
}

int aco_batch_destroy(aco_batch* b) {
  if (!b) return ACO_OK;
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  if (b->own_arena) cudaFree(b->arena_mem);
  cudaFree(b->d_insts);
  cudaFree(b->d_row_off);
  cudaFree(b->d_ant_off);
  cudaFree(b->d_ir_insts);
  cudaFree(b->d_ir_off);
  cudaFree(b->d_rw_insts);
  cudaFree(b->d_rw_off);
  cudaFree(b->d_counter);
  cudaFree(b->d_err);
  delete b;
  return ACO_OK;
}

int aco_batch_add(aco_batch* b, const float* coords_host, const aco_params* p, int iters_budget,
                  int* slot) {
  if (!b || !coords_host || !p || !slot) return set_error(ACO_ERR_ARG, "NULL argument");
  if (p->prec != b->prec) return set_error(ACO_ERR_ARG, "instance precision %d differs from the batch's %d", p->prec, b->prec);
  if (iters_budget < 0) return set_error(ACO_ERR_ARG, "iters_budget must be >= 0");
  // size errors before the arena: an instance no kernel serves is refused, not queued
  if (p->roulette == ACO_RW && p->n > kRwMaxN)
    return set_error(ACO_ERR_UNSUPPORTED, "roulette-wheel construction serves n <= %d", kRwMaxN);
  if (p->roulette != ACO_RW && p->prec == ACO_FP32 && p->n > ACO_MAX_N_FP32_BATCH)
    return set_error(ACO_ERR_UNSUPPORTED, "batched construction with fp32 M_p serves n <= %d",
                     ACO_MAX_N_FP32_BATCH);
  int q = 0;
  while (q < (int)b->slots.size() && b->slots[q].used) ++q;
  if (q == (int)b->slots.size()) return set_error(ACO_ERR_OOM, "all %d batch slots are in use", q);
  const size_t need = instance_workspace_bytes(p->n, p->m);
  size_t off = 0;
  if (p->n < 3 || p->n > ACO_MAX_N || p->m < 1) return set_error(ACO_ERR_ARG, "n or m out of range");
  if (!b->arena.alloc(need, &off))
    return set_error(ACO_ERR_OOM, "instance needs %zu bytes; arena has %zu free (largest block %zu)", need,
                     b->arena.free_bytes(), b->arena.largest());
  Slot& s = b->slots[q];
  const int rc = instance_bind(*p, b->arena_mem + off, &s.dev, b->stream, coords_host);
  if (rc) {
    b->arena.release(off);
    return rc;
  }
  s.used = true;
  s.p = *p;
  s.off = off;
  s.done = 0;
  s.budget = iters_budget;
  b->tables_ok = false;
  *slot = q;
  return ACO_OK;
}

int aco_batch_remove(aco_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
    return set_error(ACO_ERR_ARG, "invalid slot %d", slot);
  ACO_CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->arena.release(b->slots[slot].off);
  b->slots[slot] = Slot();
  b->tables_ok = false;
  return ACO_OK;
}

int aco_batch_step(aco_batch* b, int k) {
  if (!b) return set_error(ACO_ERR_ARG, "batch is NULL");
  if (k < 0) return set_error(ACO_ERR_ARG, "k must be >= 0");
  for (int q = 0; q < k; ++q) {
    if (!b->tables_ok) {
      int rc = batch_refresh(b);
      if (rc) return rc;
      if (b->active.empty()) return ACO_OK;
      rc = batch_enqueue(b);  // first iteration of a new set: direct launches
      if (rc) return rc;
    } else {
      if (b->active.empty()) return ACO_OK;
      if (!b->exec && b->stream) {
        int rc = batch_capture(b);
        if (rc) return rc;
      }
      if (b->exec) {
        ACO_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
      } else {
        int rc = batch_enqueue(b);
        if (rc) return rc;
      }
    }
    bool change = false;
    for (int id : b->active) {
      Slot& s = b->slots[id];
      s.done += 1;
      change |= s.finished();
    }
    if (change) b->tables_ok = false;
  }
  return ACO_OK;
}

int aco_batch_best(aco_batch* b, int slot, int32_t* tour_host, double* len_host) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
    return set_error(ACO_ERR_ARG, "invalid slot %d", slot);
  if (!tour_host || !len_host) return set_error(ACO_ERR_ARG, "NULL argument");
  const Slot& s = b->slots[slot];
  if (s.done == 0) return set_error(ACO_ERR_STATE, "slot %d has not run an iteration", slot);
  ACO_CUDA_TRY(cudaStreamSynchronize(b->stream));
  int32_t err = 0;
  ACO_CUDA_TRY(cudaMemcpy(&err, b->d_err, 4, cudaMemcpyDeviceToHost));
  if (err) return kernel_check_error(err);
  ACO_CUDA_TRY(cudaMemcpy(len_host, s.dev.best_len, 8, cudaMemcpyDeviceToHost));
  ACO_CUDA_TRY(cudaMemcpy(tour_host, s.dev.best_tour, sizeof(int32_t) * s.p.n, cudaMemcpyDeviceToHost));
  return ACO_OK;
}

int aco_batch_get_tau(aco_batch* b, int slot, float* tau_host) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used || !tau_host)
    return set_error(ACO_ERR_ARG, "invalid argument");
  const Slot& s = b->slots[slot];
  ACO_CUDA_TRY(cudaStreamSynchronize(b->stream));
  if (s.dev.tau_bf16) {  // bf16 storage: widened exactly to fp32
    std::vector<uint16_t> h((size_t)s.p.n * s.p.n);
    ACO_CUDA_TRY(cudaMemcpy2D(h.data(), sizeof(uint16_t) * s.p.n, s.dev.tau, sizeof(uint16_t) * s.dev.ld,
                              sizeof(uint16_t) * s.p.n, s.p.n, cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < h.size(); ++q) {
      const uint32_t bits = (uint32_t)h[q] << 16;
      std::memcpy(tau_host + q, &bits, 4);
    }
    return ACO_OK;
  }
  ACO_CUDA_TRY(cudaMemcpy2D(tau_host, sizeof(float) * s.p.n, s.dev.tau, sizeof(float) * s.dev.ld,
                            sizeof(float) * s.p.n, s.p.n, cudaMemcpyDeviceToHost));
  return ACO_OK;
}

int aco_batch_status(aco_batch* b, int slot, uint32_t* iterations_done, int* finished) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
    return set_error(ACO_ERR_ARG, "invalid slot %d", slot);
  if (iterations_done) *iterations_done = b->slots[slot].done;
  if (finished) *finished = b->slots[slot].finished() ? 1 : 0;
  return ACO_OK;
}

int aco_batch_info(aco_batch* b, int* active, size_t* free_bytes, size_t* largest_block) {
  if (!b) return set_error(ACO_ERR_ARG, "batch is NULL");
  int cnt = 0;
  for (auto& s : b->slots) cnt += s.used && !s.finished();
  if (active) *active = cnt;
  if (free_bytes) *free_bytes = b->arena.free_bytes();
  if (largest_block) *largest_block = b->arena.largest();
  return ACO_OK;
}

int aco_batch_set_shape(aco_batch* b, int warps, int chunks, int mode) {
  if (!b) return set_error(ACO_ERR_ARG, "batch is NULL");
  if (warps || chunks) {
    const int eb = b->prec == ACO_FP32 ? 4 : 2;
    const ConstructShape* list;
    const int cnt = batch_construct_shapes(eb, &list);
    bool found = false;
    for (int q = 0; q < cnt; ++q)
      found |= list[q].warps == warps && list[q].chunks == chunks && list[q].mode == mode;
    if (!found) return set_error(ACO_ERR_UNSUPPORTED, "batch shape (%d, %d, %d) not compiled", warps, chunks, mode);
  }
  b->shape = {warps, chunks, mode};
  b->tables_ok = false;
  return ACO_OK;
}

int aco_batch_instance_bytes(int n, int m, size_t* bytes) {
  if (!bytes || n < 3 || n > ACO_MAX_N || m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "invalid argument");
  *bytes = (instance_workspace_bytes(n, m) + 255) & ~(size_t)255;
  return ACO_OK;
}

}  // extern "C"
