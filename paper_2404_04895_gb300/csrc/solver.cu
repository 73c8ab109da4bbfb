// Host runtime and C ABI of the TensorACO library: solver state in device
// memory, the per-iteration launch sequence (captured once into a CUDA graph
// and replayed), the single-instance global API and the step-level calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "internal.h"
#include "steps.cuh"
#include "shapes.h"

namespace aco {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(e == cudaErrorMemoryAllocation ? ACO_ERR_OOM : ACO_ERR_CUDA, "%s: %s (%s)",
                   what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// ------------------------------------------------------------------ shapes
static const ConstructShape kShapes4[] = {
#define X(W, KC, MODE) {W, KC, MODE},
    ACO_SHAPES_4B(X)
#undef X
};
static const ConstructShape kShapes2[] = {
#define X(W, KC, MODE) {W, KC, MODE},
    ACO_SHAPES_2B(X)
#undef X
};

// The size limits of tensoraco.h are those of the compiled shapes: the
// widest covers 32 * warps * chunks * (16 / element bytes) columns.
#define ACO_WIDEST(W, KC, MODE) most = most > 32 * (W) * (KC) * V ? most : 32 * (W) * (KC) * V;
constexpr int widest_4b() { constexpr int V = 4; int most = 0; ACO_SHAPES_4B(ACO_WIDEST) return most; }
constexpr int widest_2b() { constexpr int V = 8; int most = 0; ACO_SHAPES_2B(ACO_WIDEST) return most; }
constexpr int widest_batch_4b() { constexpr int V = 4; int most = 0; ACO_BATCH_SHAPES_4B(ACO_WIDEST) return most; }
constexpr int widest_batch_2b() { constexpr int V = 8; int most = 0; ACO_BATCH_SHAPES_2B(ACO_WIDEST) return most; }
#undef ACO_WIDEST
static_assert(widest_4b() == ACO_MAX_N_FP32, "ACO_MAX_N_FP32 is the widest fp32 shape");
static_assert(widest_batch_4b() == ACO_MAX_N_FP32_BATCH, "ACO_MAX_N_FP32_BATCH is the widest fp32 batch shape");
static_assert(widest_2b() >= ACO_MAX_N && widest_batch_2b() >= ACO_MAX_N, "16-bit shapes cover ACO_MAX_N");
static_assert(kRwMaxN == ACO_MAX_N_RW && kLeanMaxN <= ACO_MAX_N_FP32_BATCH, "size limits");

static const ConstructShape kBatchShapes4[] = {
#define X(W, KC, MODE) {W, KC, MODE},
    ACO_BATCH_SHAPES_4B(X)
#undef X
};
static const ConstructShape kBatchShapes2[] = {
#define X(W, KC, MODE) {W, KC, MODE},
    ACO_BATCH_SHAPES_2B(X)
#undef X
};

int batch_construct_shapes(int elem_bytes, const ConstructShape** list) {
  if (elem_bytes == 4) {
    *list = kBatchShapes4;
    return (int)(sizeof(kBatchShapes4) / sizeof(kBatchShapes4[0]));
  }
  *list = kBatchShapes2;
  return (int)(sizeof(kBatchShapes2) / sizeof(kBatchShapes2[0]));
}

int construct_shapes(int elem_bytes, const ConstructShape** list) {
  if (elem_bytes == 4) {
    *list = kShapes4;
    return (int)(sizeof(kShapes4) / sizeof(kShapes4[0]));
  }
  *list = kShapes2;
  return (int)(sizeof(kShapes2) / sizeof(kShapes2[0]));
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, ConstructShape> g_tuned;

void register_tuned_shape(int n, int m, int elem_bytes, ConstructShape s) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[std::make_tuple(n, m, elem_bytes)] = s;
}

static int shape_columns(ConstructShape s, int elem_bytes) {
  if (s.mode == kModeLean) return kLeanMaxN;
  return 32 * s.warps * s.chunks * (16 / elem_bytes);
}

ConstructShape default_construct_shape(int n, int m, int elem_bytes) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(n, m, elem_bytes));
    if (it != g_tuned.end()) return it->second;
  }
  const ConstructShape* list;
  const int cnt = construct_shapes(elem_bytes, &list);
  ConstructShape best = {0, 0, 0};
  for (int q = 0; q < cnt; ++q) {
    const ConstructShape s = list[q];
    if (shape_columns(s, elem_bytes) < n) continue;
    const bool better = best.warps == 0 || s.mode > best.mode ||
                        (s.mode == best.mode && (s.warps < best.warps ||
                                                 (s.warps == best.warps && s.chunks < best.chunks)));
    if (better) best = s;
  }
  return best;
}

int prepare_kernels() {
  static std::once_flag once;
  static int rc = ACO_OK;
  std::call_once(once, [] {
    rc = prepare_construct_f32();
    if (!rc) rc = prepare_construct_bf16();
    if (!rc) rc = prepare_construct_f16();
    if (!rc) rc = prepare_deposit();
    if (!rc) rc = prepare_tour_length();
    if (!rc) rc = prepare_construct_lean();
    if (!rc) rc = prepare_construct_rw();
  });
  return rc == ACO_OK ? ACO_OK : set_error(rc, "kernel preparation failed");
}

static int launch_construct(const void* P, int prec, int n, int ld, int m, uint2 key, uint32_t it,
                            const uint32_t* it_dev, int32_t* tours, int32_t* err,
                            ConstructShape s, const uint2* lists, const int* lcnt,
                            const uint32_t* lkey, cudaStream_t st) {
  const int eb = prec == ACO_FP32 ? 4 : 2;
  if (s.warps == 0 && lists && n <= kLeanMaxN) s = {1, 0, kModeLean};  // lists: lean kernel by default
  if (s.warps == 0) s = default_construct_shape(n, m, eb);
  if (s.warps == 0 || shape_columns(s, eb) < n)
    return set_error(ACO_ERR_UNSUPPORTED, "no construct shape covers n=%d", n);
  if (s.mode == kModeLean)
    return launch_construct_lean(P, prec, n, ld, m, key, it, it_dev, tours, err, lists, lcnt, lkey, st);
  switch (prec) {
    case ACO_FP32:
      return launch_construct_f32(static_cast<const float*>(P), n, ld, m, key, it, it_dev, tours, err,
                                  s.warps, s.chunks, s.mode, lists, lcnt, lkey, st);
    case ACO_BF16:
      return launch_construct_bf16(P, n, ld, m, key, it, it_dev, tours, err, s.warps, s.chunks, s.mode,
                                   lists, lcnt, lkey, st);
    case ACO_FP16:
      return launch_construct_f16(P, n, ld, m, key, it, it_dev, tours, err, s.warps, s.chunks, s.mode,
                                  lists, lcnt, lkey, st);
  }
  return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
}

// ------------------------------------------------------------------ gamma
static float gamma_at(int it, int T, float gmax, float gmin) {
  if (T <= 0 || it >= T) return gmin;
  const double hi = (double)gmax, lo = (double)gmin;
  const double ang = 3.14159265358979323846 * (double)it / (double)T;
  const double g = lo + 0.5 * (hi - lo) * (1.0 + std::cos(ang));
  return (float)g;
}
static float inv_gamma_of(float g) { return (float)(1.0 / (double)g); }

// ------------------------------------------------------------------ validation
static bool is_small_int(float v) { return std::isfinite(v) && v >= 0.0f && v <= 8.0f && v == std::floor(v); }

static int validate(const aco_params* p) {
  if (!p) return set_error(ACO_ERR_ARG, "params is NULL");
  if (p->n < 3 || p->n > ACO_MAX_N) return set_error(ACO_ERR_ARG, "n=%d outside [3, %d]", p->n, ACO_MAX_N);
  if (p->m < 1 || p->m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m=%d outside [1, %d]", p->m, ACO_MAX_M);
  if (p->alpha < 0 || p->alpha > 8 || p->beta < 0 || p->beta > 8)
    return set_error(ACO_ERR_UNSUPPORTED, "alpha/beta must be integers in [0, 8]");
  if (!(p->rho >= 0.0f && p->rho <= 1.0f)) return set_error(ACO_ERR_ARG, "rho outside [0, 1]");
  if (!(p->Q > 0.0f) || !std::isfinite(p->Q)) return set_error(ACO_ERR_ARG, "Q must be finite and > 0");
  if (!(p->tau0 > 0.0f) || !std::isfinite(p->tau0)) return set_error(ACO_ERR_ARG, "tau0 must be finite and > 0");
  if (p->topk < 0) return set_error(ACO_ERR_ARG, "topk=%d must be >= 0 (0: every path deposits)", p->topk);
  if (p->tau_prec != ACO_FP32 && p->tau_prec != ACO_BF16)
    return set_error(ACO_ERR_UNSUPPORTED, "tau is stored in fp32 or bf16 (tau_prec %d)", p->tau_prec);
  if (p->tau_prec == ACO_BF16 && p->deposit != ACO_DEPOSIT_DET)
    return set_error(ACO_ERR_UNSUPPORTED, "bf16 tau needs the deterministic deposit");
  if (p->prec < ACO_FP32 || p->prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", p->prec);
  if (p->roulette != ACO_IR && p->roulette != ACO_ADAIR && p->roulette != ACO_RW)
    return set_error(ACO_ERR_ARG, "unknown roulette %d", p->roulette);
  if (p->roulette == ACO_RW && p->n > kRwMaxN)
    return set_error(ACO_ERR_UNSUPPORTED, "roulette-wheel construction serves n <= %d", kRwMaxN);
  if (p->roulette != ACO_RW && p->prec == ACO_FP32 && p->n > ACO_MAX_N_FP32)
    return set_error(ACO_ERR_UNSUPPORTED, "construction with fp32 M_p serves n <= %d", ACO_MAX_N_FP32);
  if (p->deposit != ACO_DEPOSIT_DET && p->deposit != ACO_DEPOSIT_ATOMIC)
    return set_error(ACO_ERR_ARG, "unknown deposit mode %d", p->deposit);
  if (p->roulette == ACO_ADAIR) {
    if (!(p->gamma_max > 0.0f && p->gamma_max <= 16.0f && p->gamma_min > 0.0f && p->gamma_min <= 16.0f))
      return set_error(ACO_ERR_ARG, "gamma outside (0, 16]");
    if (p->gamma_T < 1) return set_error(ACO_ERR_ARG, "gamma_T must be >= 1");
  }
  return ACO_OK;
}

// ------------------------------------------------------------------ workspace
constexpr int kSchedCap = 1 << 16;  // AdaIR schedule entries (iterations 0..T, clamped)

struct Layout {
  size_t coords, D, H, tau, P, tours, L, c, dep, nbr, best_tour, best_len, it, err, sched, lists,
      lcnt, lkey, total;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
static int ld_of(int n) { return (n + 7) & ~7; }

static Layout layout_of(int n, int m) {
  const size_t ld = (size_t)ld_of(n);
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += al(bytes);
    return at;
  };
  L.coords = take((size_t)n * 2 * 4);
  L.D = take((size_t)n * (n - 1) / 2 * 8);  // strictly upper triangle (tri_index)
  L.H = take((size_t)n * ld * 4);
  L.tau = take((size_t)n * ld * 4);
  L.P = take((size_t)n * ld * 4);
  L.tours = take((size_t)m * n * 4);
  L.L = take((size_t)m * 8);
  L.c = take((size_t)m * 8);
  L.dep = take(8);
  L.nbr = take((size_t)n * m * 2 * 4);
  // best_tour .. err adjacent: aco_solver_best reads them with one copy
  L.best_tour = take((size_t)n * 4);
  L.best_len = take(8);
  L.it = take(4);
  L.err = take(4);
  L.sched = take((size_t)kSchedCap * 4);
  L.lists = take((size_t)n * kListMax * 8);
  L.lcnt = take((size_t)n * 4);
  L.lkey = take((size_t)n * 4);
  L.total = o;
  return L;
}

size_t instance_workspace_bytes(int n, int m) { return layout_of(n, m).total; }

// Validate p, lay out an instance's state in ws (instance_workspace_bytes
// bytes, 256-byte aligned), initialise it on st (coordinates in, distances,
// eta^beta, tau = tau0, no best yet, iteration 0, AdaIR schedule) and fill d.
int instance_bind(const aco_params& p, unsigned char* ws, InstDev* d, cudaStream_t st,
                  const float* coords_host) {
  int rc = validate(&p);
  if (rc) return rc;
  for (int q = 0; q < 2 * p.n; ++q)
    if (!std::isfinite(coords_host[q])) return set_error(ACO_ERR_ARG, "coordinate %d is not finite", q);
  const Layout L = layout_of(p.n, p.m);
  const int ld = ld_of(p.n);
  InstDev x{};
  x.n = p.n;
  x.m = p.m;
  x.ld = ld;
  x.alpha = p.alpha;
  x.adair = p.roulette == ACO_ADAIR;
  x.rw = p.roulette == ACO_RW;
  x.n_sched = x.adair ? std::min(p.gamma_T + 1, kSchedCap) : 1;
  x.rho = p.rho;
  x.Q = p.Q;
  x.topk = p.topk;
  x.key = make_uint2((uint32_t)p.seed, (uint32_t)(p.seed >> 32));
  float* coords = reinterpret_cast<float*>(ws + L.coords);
  x.D = reinterpret_cast<double*>(ws + L.D);
  x.H = reinterpret_cast<float*>(ws + L.H);
  x.tau = reinterpret_cast<float*>(ws + L.tau);
  x.tau_bf16 = p.tau_prec == ACO_BF16 ? 1 : 0;
  x.P = ws + L.P;
  x.tours = reinterpret_cast<int32_t*>(ws + L.tours);
  x.L = reinterpret_cast<double*>(ws + L.L);
  x.c = reinterpret_cast<double*>(ws + L.c);
  x.dep = reinterpret_cast<int2*>(ws + L.dep);
  x.nbr = reinterpret_cast<int32_t*>(ws + L.nbr);
  x.best_tour = reinterpret_cast<int32_t*>(ws + L.best_tour);
  x.best_len = reinterpret_cast<double*>(ws + L.best_len);
  x.it = reinterpret_cast<uint32_t*>(ws + L.it);
  x.sched = reinterpret_cast<float*>(ws + L.sched);
  x.lists = p.cand_lists && !x.rw ? reinterpret_cast<uint2*>(ws + L.lists) : nullptr;
  x.lcnt = reinterpret_cast<int*>(ws + L.lcnt);
  x.lkey = reinterpret_cast<uint32_t*>(ws + L.lkey);
  ACO_CUDA_TRY(cudaMemcpyAsync(coords, coords_host, sizeof(float) * 2 * p.n, cudaMemcpyHostToDevice, st));
  rc = launch_heuristic(coords, p.n, p.beta, const_cast<double*>(x.D), const_cast<float*>(x.H), ld, true, st);
  if (!rc) rc = launch_fill_tau(x.tau, p.tau_prec, p.n, ld, p.tau0, st);
  if (rc) return rc;
  const double inf = INFINITY;
  const uint32_t zero = 0;
  ACO_CUDA_TRY(cudaMemcpyAsync(x.best_len, &inf, 8, cudaMemcpyHostToDevice, st));
  ACO_CUDA_TRY(cudaMemcpyAsync(x.it, &zero, 4, cudaMemcpyHostToDevice, st));
  ACO_CUDA_TRY(cudaMemsetAsync(x.best_tour, 0, sizeof(int32_t) * p.n, st));
  std::vector<float> h((size_t)x.n_sched, 1.0f);
  if (x.adair)
    for (int q = 0; q < x.n_sched; ++q) h[q] = inv_gamma_of(gamma_at(q, p.gamma_T, p.gamma_max, p.gamma_min));
  ACO_CUDA_TRY(cudaMemcpyAsync(const_cast<float*>(x.sched), h.data(), sizeof(float) * x.n_sched,
                               cudaMemcpyHostToDevice, st));
  ACO_CUDA_TRY(cudaStreamSynchronize(st));  // pageable sources above
  *d = x;
  return ACO_OK;
}

}  // namespace aco

using namespace aco;

struct aco_solver {
  aco_params p;
  int ld;
  cudaStream_t stream;
  bool own_ws;
  unsigned char* ws;
  Layout lay;
  float *coords, *H, *tau, *P_f, *sched;
  uint2* lists;
  int* lcnt;
  uint32_t* lkey;
  double *D, *L, *c, *best_len;
  int2* dep;
  int32_t *tours, *nbr, *best_tour, *err;
  uint32_t* it_dev;
  uint32_t it;                 // iterations completed (host mirror)
  ConstructShape shape;        // {0,0}: default for (n, m, prec)
  uint32_t wait_polls;         // bound on the roulette-wheel kernel's row-copy waits
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool graph_ok;
  bool use_graph;
  bool P_cur;                  // M_p and its lists are those of the current tau and iteration
  bool profiling;
  cudaEvent_t ev[7];           // probes around the iteration's kernels
  unsigned char* stage;        // pinned host copy of best_tour .. err (aco_solver_best)

  template <class T>
  T* at(size_t off) { return reinterpret_cast<T*>(ws + off); }
};

namespace aco {

static int upload_schedule(aco_solver* s) {
  const aco_params& p = s->p;
  if (p.roulette != ACO_ADAIR) return ACO_OK;
  const int cnt = std::min(p.gamma_T + 1, kSchedCap);
  std::vector<float> h((size_t)cnt);
  for (int q = 0; q < cnt; ++q) h[q] = inv_gamma_of(gamma_at(q, p.gamma_T, p.gamma_max, p.gamma_min));
  ACO_CUDA_TRY(cudaMemcpyAsync(s->sched, h.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice, s->stream));
  // pageable copy: make it complete before the host buffer goes away
  ACO_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return ACO_OK;
}

// Every change of a solver's parameters or state drops its graph; M_p is
// then no longer assumed current either.
static void drop_graph(aco_solver* s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->exec = nullptr;
  s->graph = nullptr;
  s->graph_ok = false;
  s->P_cur = false;
}

// With candidate lists and the deterministic deposit, an iteration's M_p and
// lists are computed at the end of the iteration before it, by the fused
// deposit (deposit_P_lists_kernel), which re-reads each tau row right after
// writing it; the first iteration after creation or any change computes
// them first (ensure_P).
static bool fused_P(const aco_solver* s) {
  return s->p.cand_lists != 0 && s->p.roulette != ACO_RW && s->p.deposit == ACO_DEPOSIT_DET;
}

// The launches of one iteration (a)-(d); the iteration number and AdaIR's
// exponent are read from device memory so the sequence can be replayed.
static int enqueue_iteration(aco_solver* s) {
  const aco_params& p = s->p;
  const int n = p.n, m = p.m;
  cudaStream_t st = s->stream;
  const int n_sched = std::min(p.gamma_T + 1, kSchedCap);
  // External records become event nodes of the captured graph, so the probes
  // time every replay of it (a plain record only orders captured work).
  auto probe = [&](int q) {
    if (s->profiling) cudaEventRecordWithFlags(s->ev[q], st, cudaEventRecordExternal);
  };
  probe(0);
  const bool rw = p.roulette == ACO_RW;
  const bool lists = p.cand_lists != 0 && !rw;
  const bool fused = fused_P(s);
  const float* sched = p.roulette == ACO_ADAIR ? s->sched : nullptr;
  // with lists: M_p and its lists in one pass (the probe between them then
  // gives the list step 0 ms); fused: computed by the iteration before
  int rc = ACO_OK;
  if (!fused)
    rc = lists ? launch_build_P_lists(s->tau, p.tau_prec, s->H, n, s->ld, p.alpha, 1.0f, sched, s->it_dev, n_sched,
                                      p.rho, p.prec, s->P_f, s->lists, s->lcnt, s->lkey, st)
               : launch_build_P(s->tau, p.tau_prec, s->H, n, s->ld, p.alpha, 1.0f, sched, s->it_dev, n_sched, p.prec,
                                s->P_f, st);
  if (rc) return rc;
  probe(1);
  probe(2);
  const uint2 key = make_uint2((uint32_t)p.seed, (uint32_t)(p.seed >> 32));
  if (rw)
    rc = launch_construct_rw(s->P_f, p.prec, n, s->ld, m, key, 0u, s->it_dev, s->tours, s->err, s->wait_polls, st);
  else
    rc = launch_construct(s->P_f, p.prec, n, s->ld, m, key, 0u, s->it_dev, s->tours, s->err, s->shape,
                          lists ? s->lists : nullptr, s->lcnt, s->lkey, st);
  if (rc) return rc;
  probe(3);
  const bool det = p.deposit == ACO_DEPOSIT_DET;
  rc = launch_tour_length(s->D, n, s->tours, m, p.Q, s->L, s->c, det ? s->nbr : nullptr, true, st);
  if (rc) return rc;
  probe(4);
  rc = launch_best(s->L, s->tours, n, m, s->best_tour, s->best_len, s->it_dev, s->c, p.topk,
                   det ? s->dep : nullptr, s->err, st);
  if (rc) return rc;
  probe(5);
  if (fused)  // the deposit, then the next iteration's M_p and lists
    rc = launch_deposit_P_lists(s->tau, p.tau_prec, n, s->ld, s->nbr, s->c, m, p.rho, s->dep, s->H, p.alpha, sched,
                                s->it_dev, n_sched, p.prec, s->P_f, s->lists, s->lcnt, s->lkey, st);
  else if (det)
    rc = launch_deposit(s->tau, p.tau_prec, n, s->ld, s->nbr, s->c, m, p.rho, s->dep, s->err, st);
  else
    rc = launch_deposit_atomic(s->tau, n, s->ld, s->tours, s->c, m, p.rho, st);
  if (rc) return rc;
  probe(6);
  return ACO_OK;
}

// M_p and its lists for the current tau and iteration, when the fused
// deposit did not leave them (fused mode only; queued on the solver's stream).
static int ensure_P(aco_solver* s) {
  if (!fused_P(s) || s->P_cur) return ACO_OK;
  const aco_params& p = s->p;
  const int n_sched = std::min(p.gamma_T + 1, kSchedCap);
  const float* sched = p.roulette == ACO_ADAIR ? s->sched : nullptr;
  const int rc = launch_build_P_lists(s->tau, p.tau_prec, s->H, p.n, s->ld, p.alpha, 1.0f, sched, s->it_dev, n_sched,
                                      p.rho, p.prec, s->P_f, s->lists, s->lcnt, s->lkey, s->stream);
  if (rc) return rc;
  s->P_cur = true;
  return ACO_OK;
}

static int build_graph(aco_solver* s) {
  drop_graph(s);
  ACO_CUDA_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_iteration(s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s->stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&s->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_error(e, "cudaGraphInstantiate");
  }
  s->graph = g;
  s->graph_ok = true;
  return ACO_OK;
}

// The host's reading of an error word the kernels set: a wait that ran out
// is ACO_ERR_TIMEOUT, any other check ACO_ERR_CUDA.
int kernel_check_error(int32_t code) {
  if (code == kErrTimeout)
    return set_error(ACO_ERR_TIMEOUT, "a bounded device-side wait ran out (code %d)", code);
  return set_error(ACO_ERR_CUDA, "a kernel-side check failed (code %d)", code);
}

// Waits for the solver's work and reports a kernel-side check once: the
// error word is cleared when it is read, so the solver stays usable (its
// state after a failed iteration is not meaningful; restore a checkpoint).
static int solver_sync_check(aco_solver* s) {
  ACO_CUDA_TRY(cudaStreamSynchronize(s->stream));
  int32_t err = 0;
  ACO_CUDA_TRY(cudaMemcpy(&err, s->err, 4, cudaMemcpyDeviceToHost));
  if (!err) return ACO_OK;
  ACO_CUDA_TRY(cudaMemset(s->err, 0, 4));
  return kernel_check_error(err);
}

}  // namespace aco

static int check_mat(const void* p, int n, int ld, const char* name) {
  if (!p) return set_error(ACO_ERR_ARG, "%s is NULL", name);
  if (n < 3 || n > ACO_MAX_N) return set_error(ACO_ERR_ARG, "n=%d outside [3, %d]", n, ACO_MAX_N);
  if (ld < n || (ld & 7)) return set_error(ACO_ERR_ARG, "ld=%d must be >= n and a multiple of 8", ld);
  if (!aligned16(p)) return set_error(ACO_ERR_ARG, "%s must be 16-byte aligned", name);
  return ACO_OK;
}

// ====================================================================== C ABI
extern "C" {

const char* aco_last_error(void) { return g_err; }

int aco_params_default(aco_params* p) {
  if (!p) return set_error(ACO_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->alpha = 1;
  p->beta = 2;
  p->rho = 0.5f;
  p->Q = 1.0f;
  p->tau0 = 1.0f;
  p->prec = ACO_FP32;
  p->roulette = ACO_IR;
  p->deposit = ACO_DEPOSIT_DET;
  p->gamma_max = 1.5f;
  p->gamma_min = 0.5f;
  p->gamma_T = 100;
  p->cand_lists = 1;
  p->topk = 0;
  return ACO_OK;
}

int aco_workspace_bytes(int n, int m, int prec, size_t* bytes) {
  if (!bytes) return set_error(ACO_ERR_ARG, "bytes is NULL");
  if (n < 3 || n > ACO_MAX_N || m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "n or m out of range");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  *bytes = layout_of(n, m).total;
  return ACO_OK;
}

int aco_create(aco_solver** out, const float* coords_host, const aco_params* p, void* dev_workspace,
               size_t ws_bytes, void* stream) {
  if (!out || !coords_host) return set_error(ACO_ERR_ARG, "NULL argument");
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  for (int q = 0; q < 2 * p->n; ++q)
    if (!std::isfinite(coords_host[q])) return set_error(ACO_ERR_ARG, "coordinate %d is not finite", q);
  rc = prepare_kernels();
  if (rc) return rc;
  aco_solver* s = new aco_solver();
  s->p = *p;
  s->wait_polls = kRwWaitPolls;
  s->ld = ld_of(p->n);
  s->stream = static_cast<cudaStream_t>(stream);
  s->lay = layout_of(p->n, p->m);
  if (dev_workspace) {
    if (ws_bytes < s->lay.total) {
      delete s;
      return set_error(ACO_ERR_OOM, "workspace of %zu bytes < %zu needed", ws_bytes, s->lay.total);
    }
    if (((uintptr_t)dev_workspace & 255u) != 0) {
      delete s;
      return set_error(ACO_ERR_ARG, "workspace must be 256-byte aligned");
    }
    s->ws = static_cast<unsigned char*>(dev_workspace);
    s->own_ws = false;
  } else {
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, s->lay.total);
    if (e != cudaSuccess) {
      delete s;
      return cuda_error(e, "cudaMalloc(workspace)");
    }
    s->ws = static_cast<unsigned char*>(mem);
    s->own_ws = true;
  }
  {
    const cudaError_t e = cudaMallocHost(&s->stage, s->lay.err + 4 - s->lay.best_tour);
    if (e != cudaSuccess) {
      if (s->own_ws) cudaFree(s->ws);
      delete s;
      return cuda_error(e, "cudaMallocHost(result staging)");
    }
  }
  const Layout& L = s->lay;
  s->coords = s->at<float>(L.coords);
  s->D = s->at<double>(L.D);
  s->H = s->at<float>(L.H);
  s->tau = s->at<float>(L.tau);
  s->P_f = s->at<float>(L.P);
  s->tours = s->at<int32_t>(L.tours);
  s->L = s->at<double>(L.L);
  s->c = s->at<double>(L.c);
  s->dep = s->at<int2>(L.dep);
  s->nbr = s->at<int32_t>(L.nbr);
  s->best_tour = s->at<int32_t>(L.best_tour);
  s->best_len = s->at<double>(L.best_len);
  s->it_dev = s->at<uint32_t>(L.it);
  s->err = s->at<int32_t>(L.err);
  s->sched = s->at<float>(L.sched);
  s->lists = s->at<uint2>(L.lists);
  s->lcnt = s->at<int>(L.lcnt);
  s->lkey = s->at<uint32_t>(L.lkey);
  // Replay through a CUDA graph on a created stream; the legacy default stream
  // cannot be captured, so there the iteration's kernels are launched directly.
  s->use_graph = s->stream != nullptr;

  auto fail = [&](int code) {
    drop_graph(s);
    if (s->own_ws) cudaFree(s->ws);
    cudaFreeHost(s->stage);
    delete s;
    return code;
  };
  const int n = p->n;
  cudaStream_t st = s->stream;
  if (cudaMemcpyAsync(s->coords, coords_host, sizeof(float) * 2 * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(cuda_error(cudaGetLastError(), "copy coords"));
  rc = launch_heuristic(s->coords, n, p->beta, s->D, s->H, s->ld, true, st);
  if (!rc) rc = launch_fill_tau(s->tau, p->tau_prec, n, s->ld, p->tau0, st);
  if (rc) return fail(rc);
  const double inf = INFINITY;
  const uint32_t zero = 0;
  if (cudaMemcpyAsync(s->best_len, &inf, 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->it_dev, &zero, 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(s->err, 0, 4, st) != cudaSuccess ||
      cudaMemsetAsync(s->best_tour, 0, sizeof(int32_t) * n, st) != cudaSuccess)
    return fail(cuda_error(cudaGetLastError(), "initialise state"));
  rc = upload_schedule(s);
  if (rc) return fail(rc);
  if (s->use_graph) {  // capture the iteration on the host while the set-up kernels run
    rc = build_graph(s);
    if (rc) return fail(rc);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(cuda_error(cudaGetLastError(), "init sync"));
  *out = s;
  return ACO_OK;
}

int aco_destroy(aco_solver* s) {
  if (!s) return ACO_OK;
  cudaStreamSynchronize(s->stream);
  drop_graph(s);
  if (s->profiling)
    for (int q = 0; q < 7; ++q) cudaEventDestroy(s->ev[q]);
  if (s->own_ws) cudaFree(s->ws);
  cudaFreeHost(s->stage);
  delete s;
  return ACO_OK;
}

int aco_solver_iterate(aco_solver* s, int k) {
  if (!s) return set_error(ACO_ERR_ARG, "solver is NULL");
  if (k < 0) return set_error(ACO_ERR_ARG, "k must be >= 0");
  for (int q = 0; q < k; ++q) {
    if (s->use_graph) {
      if (!s->graph_ok) {
        int rc = build_graph(s);
        if (rc) return rc;
      }
      int rc = ensure_P(s);
      if (rc) return rc;
      ACO_CUDA_TRY(cudaGraphLaunch(s->exec, s->stream));
    } else {
      int rc = ensure_P(s);
      if (!rc) rc = enqueue_iteration(s);
      if (rc) return rc;
    }
    s->it += 1;
  }
  return ACO_OK;
}

int aco_solver_best(aco_solver* s, int32_t* tour_host, double* len_host) {
  if (!s || !tour_host || !len_host) return set_error(ACO_ERR_ARG, "NULL argument");
  if (s->it == 0) return set_error(ACO_ERR_STATE, "no iteration has run yet");
  // best tour, best length and the error word in one copy after the solver's work
  const Layout& L = s->lay;
  ACO_CUDA_TRY(cudaMemcpyAsync(s->stage, s->ws + L.best_tour, L.err + 4 - L.best_tour, cudaMemcpyDeviceToHost,
                               s->stream));
  ACO_CUDA_TRY(cudaStreamSynchronize(s->stream));
  int32_t err = 0;
  std::memcpy(&err, s->stage + (L.err - L.best_tour), 4);
  if (err) {  // reported once, as solver_sync_check does
    ACO_CUDA_TRY(cudaMemset(s->err, 0, 4));
    return kernel_check_error(err);
  }
  std::memcpy(len_host, s->stage + (L.best_len - L.best_tour), 8);
  std::memcpy(tour_host, s->stage, sizeof(int32_t) * s->p.n);
  return ACO_OK;
}

// tau (n x n, dense fp32) from the device, whatever its storage
static int copy_tau_out(aco_solver* s, float* tau_host) {
  const int n = s->p.n;
  if (s->p.tau_prec != ACO_BF16) {
    ACO_CUDA_TRY(cudaMemcpy2D(tau_host, sizeof(float) * n, s->tau, sizeof(float) * s->ld, sizeof(float) * n, n,
                              cudaMemcpyDeviceToHost));
    return ACO_OK;
  }
  std::vector<uint16_t> h((size_t)n * n);
  ACO_CUDA_TRY(cudaMemcpy2D(h.data(), sizeof(uint16_t) * n, s->tau, sizeof(uint16_t) * s->ld,
                            sizeof(uint16_t) * n, n, cudaMemcpyDeviceToHost));
  for (size_t q = 0; q < h.size(); ++q) {
    const uint32_t b = (uint32_t)h[q] << 16;
    std::memcpy(tau_host + q, &b, 4);
  }
  return ACO_OK;
}

// tau to the device (dense fp32 host values; bf16 storage takes their high halves,
// exact for values that came from bf16)
static int copy_tau_in(aco_solver* s, const float* tau_host) {
  const int n = s->p.n;
  if (s->p.tau_prec != ACO_BF16) {
    ACO_CUDA_TRY(cudaMemcpy2D(s->tau, sizeof(float) * s->ld, tau_host, sizeof(float) * n, sizeof(float) * n, n,
                              cudaMemcpyHostToDevice));
    return ACO_OK;
  }
  std::vector<uint16_t> h((size_t)n * n);
  for (size_t q = 0; q < h.size(); ++q) {
    uint32_t b;
    std::memcpy(&b, tau_host + q, 4);
    if (b & 0xFFFFu) return set_error(ACO_ERR_ARG, "tau entry %zu is not a bfloat16 value", q);
    h[q] = (uint16_t)(b >> 16);
  }
  ACO_CUDA_TRY(cudaMemcpy2D(s->tau, sizeof(uint16_t) * s->ld, h.data(), sizeof(uint16_t) * n,
                            sizeof(uint16_t) * n, n, cudaMemcpyHostToDevice));
  return ACO_OK;
}

int aco_solver_get_tau(aco_solver* s, float* tau_host) {
  if (!s || !tau_host) return set_error(ACO_ERR_ARG, "NULL argument");
  int rc = solver_sync_check(s);
  if (rc) return rc;
  return copy_tau_out(s, tau_host);
}

int aco_solver_get_tours(aco_solver* s, int32_t* tours_host) {
  if (!s || !tours_host) return set_error(ACO_ERR_ARG, "NULL argument");
  int rc = solver_sync_check(s);
  if (rc) return rc;
  ACO_CUDA_TRY(cudaMemcpy(tours_host, s->tours, sizeof(int32_t) * s->p.m * s->p.n, cudaMemcpyDeviceToHost));
  return ACO_OK;
}

int aco_solver_get_lengths(aco_solver* s, double* lengths_host) {
  if (!s || !lengths_host) return set_error(ACO_ERR_ARG, "NULL argument");
  int rc = solver_sync_check(s);
  if (rc) return rc;
  ACO_CUDA_TRY(cudaMemcpy(lengths_host, s->L, sizeof(double) * s->p.m, cudaMemcpyDeviceToHost));
  return ACO_OK;
}

int aco_solver_device_state(aco_solver* s, float** tau, int* ld, int32_t** tours, double** lengths,
                            int32_t** best_tour, double** best_len) {
  if (!s) return set_error(ACO_ERR_ARG, "solver is NULL");
  if (tau) *tau = s->tau;
  if (ld) *ld = s->ld;
  if (tours) *tours = s->tours;
  if (lengths) *lengths = s->L;
  if (best_tour) *best_tour = s->best_tour;
  if (best_len) *best_len = s->best_len;
  return ACO_OK;
}

// ------------------------------------------------------------------ checkpoints
// Blob: header, tau (fp32 n x n, dense), best tour (int32 n), FNV-1a 64 of
// everything before it.  Everything else of the state is derived: M_p and the
// lists from tau each iteration, distances and eta^beta from the coordinates,
// random numbers from (seed, iteration, ant, step), so a restored run
// continues bit for bit.
namespace {
struct CkptHeader {
  char magic[8];      // "TACOCKP1"
  uint32_t version;   // 1
  uint32_t header_bytes;
  aco_params params;  // must equal the restoring solver's
  uint32_t it;
  uint32_t has_best;
  double best_len;
};

uint64_t fnv1a(const unsigned char* p, size_t bytes) {
  uint64_t h = 1469598103934665603ull;
  for (size_t q = 0; q < bytes; ++q) {
    h ^= p[q];
    h *= 1099511628211ull;
  }
  return h;
}

size_t ckpt_bytes(int n) {
  return sizeof(CkptHeader) + sizeof(float) * (size_t)n * n + sizeof(int32_t) * (size_t)n + sizeof(uint64_t);
}

bool same_params(const aco_params& a, const aco_params& b) {
  return a.n == b.n && a.m == b.m && a.alpha == b.alpha && a.beta == b.beta && a.rho == b.rho && a.Q == b.Q &&
         a.tau0 == b.tau0 && a.seed == b.seed && a.prec == b.prec && a.roulette == b.roulette &&
         a.deposit == b.deposit && a.gamma_max == b.gamma_max && a.gamma_min == b.gamma_min &&
         a.gamma_T == b.gamma_T && a.topk == b.topk && a.tau_prec == b.tau_prec;
}
}  // namespace

int aco_solver_state_bytes(aco_solver* s, size_t* bytes) {
  if (!s || !bytes) return set_error(ACO_ERR_ARG, "NULL argument");
  *bytes = ckpt_bytes(s->p.n);
  return ACO_OK;
}

int aco_solver_save(aco_solver* s, void* host_buf, size_t bytes) {
  if (!s || !host_buf) return set_error(ACO_ERR_ARG, "NULL argument");
  const int n = s->p.n;
  if (bytes < ckpt_bytes(n)) return set_error(ACO_ERR_ARG, "buffer holds %zu bytes; the state needs %zu", bytes, ckpt_bytes(n));
  int rc = solver_sync_check(s);
  if (rc) return rc;
  unsigned char* out = static_cast<unsigned char*>(host_buf);
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "TACOCKP1", 8);
  h.version = 1;
  h.header_bytes = (uint32_t)sizeof(CkptHeader);
  h.params = s->p;
  h.it = s->it;
  h.has_best = s->it > 0;
  ACO_CUDA_TRY(cudaMemcpy(&h.best_len, s->best_len, 8, cudaMemcpyDeviceToHost));
  std::memcpy(out, &h, sizeof(h));
  float* tau = reinterpret_cast<float*>(out + sizeof(h));
  rc = copy_tau_out(s, tau);
  if (rc) return rc;
  int32_t* best = reinterpret_cast<int32_t*>(tau + (size_t)n * n);
  ACO_CUDA_TRY(cudaMemcpy(best, s->best_tour, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  const size_t body = ckpt_bytes(n) - sizeof(uint64_t);
  const uint64_t sum = fnv1a(out, body);
  std::memcpy(out + body, &sum, sizeof(sum));
  return ACO_OK;
}

int aco_solver_load(aco_solver* s, const void* host_buf, size_t bytes) {
  if (!s || !host_buf) return set_error(ACO_ERR_ARG, "NULL argument");
  const int n = s->p.n;
  if (bytes != ckpt_bytes(n)) return set_error(ACO_ERR_ARG, "checkpoint has %zu bytes; this solver's state has %zu", bytes, ckpt_bytes(n));
  const unsigned char* in = static_cast<const unsigned char*>(host_buf);
  CkptHeader h;
  std::memcpy(&h, in, sizeof(h));
  if (std::memcmp(h.magic, "TACOCKP1", 8) != 0 || h.version != 1 || h.header_bytes != sizeof(CkptHeader))
    return set_error(ACO_ERR_ARG, "not a checkpoint of this format");
  const size_t body = ckpt_bytes(n) - sizeof(uint64_t);
  uint64_t sum = 0;
  std::memcpy(&sum, in + body, sizeof(sum));
  if (sum != fnv1a(in, body)) return set_error(ACO_ERR_ARG, "checkpoint checksum mismatch (corrupted)");
  if (!same_params(h.params, s->p)) return set_error(ACO_ERR_ARG, "checkpoint parameters differ from the solver's");
  int rc = solver_sync_check(s);
  if (rc) return rc;
  const float* tau = reinterpret_cast<const float*>(in + sizeof(h));
  for (size_t q = 0; q < (size_t)n * n; ++q)
    if (!(tau[q] >= 0.0f)) return set_error(ACO_ERR_ARG, "checkpoint tau entry %zu is negative or NaN", q);
  const int32_t* best = reinterpret_cast<const int32_t*>(tau + (size_t)n * n);
  rc = copy_tau_in(s, tau);
  if (rc) return rc;
  ACO_CUDA_TRY(cudaMemcpy(s->best_tour, best, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  const double bl = h.has_best ? h.best_len : INFINITY;
  ACO_CUDA_TRY(cudaMemcpy(s->best_len, &bl, 8, cudaMemcpyHostToDevice));
  ACO_CUDA_TRY(cudaMemcpy(s->it_dev, &h.it, 4, cudaMemcpyHostToDevice));
  s->it = h.it;
  return ACO_OK;
}

int aco_solver_iteration(aco_solver* s, uint32_t* it) {
  if (!s || !it) return set_error(ACO_ERR_ARG, "NULL argument");
  *it = s->it;
  return ACO_OK;
}

int aco_solver_set_profiling(aco_solver* s, int on) {
  if (!s) return set_error(ACO_ERR_ARG, "solver is NULL");
  if ((bool)on == s->profiling) return ACO_OK;
  ACO_CUDA_TRY(cudaStreamSynchronize(s->stream));
  drop_graph(s);
  if (on) {
    for (int q = 0; q < 7; ++q) ACO_CUDA_TRY(cudaEventCreate(&s->ev[q]));
  } else {
    for (int q = 0; q < 7; ++q) cudaEventDestroy(s->ev[q]);
  }
  s->profiling = on != 0;
  return ACO_OK;
}

int aco_solver_kernel_ms(aco_solver* s, float* ms6) {
  if (!s || !ms6) return set_error(ACO_ERR_ARG, "NULL argument");
  if (!s->profiling) return set_error(ACO_ERR_STATE, "profiling is off");
  if (s->it == 0) return set_error(ACO_ERR_STATE, "no iteration has run yet");
  ACO_CUDA_TRY(cudaEventSynchronize(s->ev[6]));
  for (int q = 0; q < 6; ++q) ACO_CUDA_TRY(cudaEventElapsedTime(&ms6[q], s->ev[q], s->ev[q + 1]));
  return ACO_OK;
}

int aco_solver_set_wait_polls(aco_solver* s, uint32_t polls) {
  if (!s) return set_error(ACO_ERR_ARG, "solver is NULL");
  s->wait_polls = polls;
  drop_graph(s);  // the bound is a launch argument of the captured graph
  return ACO_OK;
}

int aco_solver_set_shape(aco_solver* s, int warps, int chunks, int mode) {
  if (!s) return set_error(ACO_ERR_ARG, "solver is NULL");
  if (warps || chunks) {
    const int eb = s->p.prec == ACO_FP32 ? 4 : 2;
    const ConstructShape* list;
    const int cnt = construct_shapes(eb, &list);
    bool found = mode == kModeLean && warps == 1;
    for (int q = 0; q < cnt; ++q)
      found |= list[q].warps == warps && list[q].chunks == chunks && list[q].mode == mode;
    if (!found) return set_error(ACO_ERR_UNSUPPORTED, "shape (%d, %d, %d) not compiled", warps, chunks, mode);
    if (shape_columns({warps, chunks, mode}, eb) < s->p.n)
      return set_error(ACO_ERR_ARG, "shape (%d, %d) does not cover n=%d", warps, chunks, s->p.n);
  }
  s->shape = {warps, chunks, mode};
  drop_graph(s);
  return ACO_OK;
}

int aco_autotune_construct(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed,
                           int32_t* tours_scratch_dev, int reps, int* warps_out, int* chunks_out,
                           int* mode_out, float* ms_out, void* stream) {
  int rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (!tours_scratch_dev || m < 1 || m > ACO_MAX_M || reps < 1) return set_error(ACO_ERR_ARG, "invalid argument");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  rc = prepare_kernels();
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int eb = prec == ACO_FP32 ? 4 : 2;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const ConstructShape* list;
  const int cnt = construct_shapes(eb, &list);
  cudaEvent_t e0, e1;
  ACO_CUDA_TRY(cudaEventCreate(&e0));
  ACO_CUDA_TRY(cudaEventCreate(&e1));
  ConstructShape best = {0, 0, 0};
  float best_ms = 0.0f;
  for (int q = 0; q < cnt && rc == ACO_OK; ++q) {
    if (shape_columns(list[q], eb) < n) continue;
    rc = launch_construct(P_dev, prec, n, ld, m, key, 0u, nullptr, tours_scratch_dev, nullptr, list[q],
                          nullptr, nullptr, nullptr, st);
    if (rc) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && rc == ACO_OK; ++r)
      rc = launch_construct(P_dev, prec, n, ld, m, key, (uint32_t)(r + 1), nullptr, tours_scratch_dev,
                            nullptr, list[q], nullptr, nullptr, nullptr, st);
    cudaEventRecord(e1, st);
    if (rc) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = cuda_error(cudaGetLastError(), "autotune sync");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (best.warps == 0 || ms < best_ms) {
      best = list[q];
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best.warps == 0) return set_error(ACO_ERR_UNSUPPORTED, "no construct shape covers n=%d", n);
  register_tuned_shape(n, m, eb, best);
  if (warps_out) *warps_out = best.warps;
  if (chunks_out) *chunks_out = best.chunks;
  if (mode_out) *mode_out = best.mode;
  if (ms_out) *ms_out = best_ms;
  return ACO_OK;
}

// ---------------------------------------------------------------- global API
static aco_solver* g_solver = nullptr;
static void* g_ws = nullptr;
static size_t g_ws_bytes = 0;
static void* g_stream = nullptr;
// The global solver's stream when none is bound: created on first use, kept
// for the process.  A created stream (unlike the legacy default stream) can
// be captured, so the global solver's iterations replay as one graph.
static cudaStream_t g_own_stream = nullptr;
static aco_params g_pending = [] {
  aco_params p;
  aco_params_default(&p);
  return p;
}();

int aco_bind(void* dev_workspace, size_t bytes, void* stream) {
  g_ws = dev_workspace;
  g_ws_bytes = dev_workspace ? bytes : 0;
  g_stream = stream;
  return ACO_OK;
}

int aco_init(const float* coords_host, int n, int m, float alpha, float beta, float rho, float Q,
             uint64_t seed) {
  if (!is_small_int(alpha) || !is_small_int(beta))
    return set_error(ACO_ERR_UNSUPPORTED, "alpha and beta must be integers in [0, 8]");
  aco_params p = g_pending;
  p.n = n;
  p.m = m;
  p.alpha = (int)alpha;
  p.beta = (int)beta;
  p.rho = rho;
  p.Q = Q;
  p.seed = seed;
  if (g_solver) {
    aco_destroy(g_solver);
    g_solver = nullptr;
  }
  void* stream = g_stream;
  if (!stream) {
    if (!g_own_stream) {
      const cudaError_t e = cudaStreamCreate(&g_own_stream);
      if (e != cudaSuccess) {
        g_own_stream = nullptr;
        return cuda_error(e, "cudaStreamCreate");
      }
    }
    stream = g_own_stream;
  }
  return aco_create(&g_solver, coords_host, &p, g_ws, g_ws_bytes, stream);
}

int aco_set_variant(int roulette, float gamma_max, float gamma_min, int T) {
  aco_params p = g_solver ? g_solver->p : g_pending;
  p.roulette = roulette;
  p.gamma_max = gamma_max;
  p.gamma_min = gamma_min;
  p.gamma_T = T;
  if (p.n == 0) {  // no solver yet: validate the variant fields only
    if (roulette != ACO_IR && roulette != ACO_ADAIR && roulette != ACO_RW)
      return set_error(ACO_ERR_ARG, "unknown roulette %d", roulette);
    if (roulette == ACO_ADAIR && (!(gamma_max > 0 && gamma_max <= 16 && gamma_min > 0 && gamma_min <= 16) || T < 1))
      return set_error(ACO_ERR_ARG, "invalid gamma schedule");
  } else {
    int rc = validate(&p);
    if (rc) return rc;
  }
  g_pending.roulette = roulette;
  g_pending.gamma_max = gamma_max;
  g_pending.gamma_min = gamma_min;
  g_pending.gamma_T = T;
  if (g_solver) {
    g_solver->p = p;
    drop_graph(g_solver);
    return upload_schedule(g_solver);
  }
  return ACO_OK;
}

int aco_set_precision(int prec) {
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  if (g_solver) {
    aco_params p = g_solver->p;
    p.prec = prec;
    const int rc = validate(&p);
    if (rc) return rc;
  }
  g_pending.prec = prec;
  if (g_solver) {
    g_solver->p.prec = prec;
    drop_graph(g_solver);
  }
  return ACO_OK;
}

int aco_set_tau_precision(int prec) {
  if (prec != ACO_FP32 && prec != ACO_BF16) return set_error(ACO_ERR_UNSUPPORTED, "tau is stored in fp32 or bf16");
  g_pending.tau_prec = prec;
  return ACO_OK;
}

int aco_set_deposit_topk(int k) {
  if (k < 0) return set_error(ACO_ERR_ARG, "topk=%d must be >= 0 (0: every path deposits)", k);
  g_pending.topk = k;
  if (g_solver) {
    g_solver->p.topk = k;
    drop_graph(g_solver);
  }
  return ACO_OK;
}

int aco_op_select_topk(const double* L_dev, int m, int k, double* c_dev, void* stream) {
  if (!L_dev || !c_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m out of range");
  return launch_select_topk(L_dev, m, k, c_dev, static_cast<cudaStream_t>(stream));
}

int aco_set_deposit(int mode) {
  if (mode != ACO_DEPOSIT_DET && mode != ACO_DEPOSIT_ATOMIC) return set_error(ACO_ERR_ARG, "unknown deposit mode %d", mode);
  g_pending.deposit = mode;
  if (g_solver) {
    g_solver->p.deposit = mode;
    drop_graph(g_solver);
  }
  return ACO_OK;
}

#define ACO_NEED_SOLVER() \
  if (!g_solver) return set_error(ACO_ERR_STATE, "aco_init has not been called")

int aco_iterate(int k) {
  ACO_NEED_SOLVER();
  return aco_solver_iterate(g_solver, k);
}
int aco_best(int32_t* tour, double* len) {
  ACO_NEED_SOLVER();
  return aco_solver_best(g_solver, tour, len);
}
int aco_get_tau(float* tau) {
  ACO_NEED_SOLVER();
  return aco_solver_get_tau(g_solver, tau);
}
int aco_get_tours(int32_t* tours) {
  ACO_NEED_SOLVER();
  return aco_solver_get_tours(g_solver, tours);
}
int aco_get_lengths(double* L) {
  ACO_NEED_SOLVER();
  return aco_solver_get_lengths(g_solver, L);
}
int aco_free(void) {
  int rc = aco_destroy(g_solver);
  g_solver = nullptr;
  return rc;
}

// ---------------------------------------------------------------- step-level API

int aco_op_heuristic(const float* coords_dev, int n, int beta, double* D_dev, float* H_dev, int ld,
                     void* stream) {
  int rc = check_mat(H_dev, n, ld, "H");
  if (rc) return rc;
  if (!coords_dev) return set_error(ACO_ERR_ARG, "coords is NULL");
  if (beta < 0 || beta > 8) return set_error(ACO_ERR_UNSUPPORTED, "beta must be an integer in [0, 8]");
  return launch_heuristic(coords_dev, n, beta, D_dev, H_dev, ld, false, static_cast<cudaStream_t>(stream));
}

int aco_op_fill(float* dev, int n, int ld, float value, void* stream) {
  int rc = check_mat(dev, n, ld, "matrix");
  if (rc) return rc;
  return launch_fill(dev, n, ld, value, static_cast<cudaStream_t>(stream));
}

int aco_op_build_P(const float* tau_dev, const float* H_dev, int n, int ld, int alpha, float inv_gamma,
                   int prec, void* P_dev, void* stream) {
  int rc = check_mat(tau_dev, n, ld, "tau");
  if (!rc) rc = check_mat(H_dev, n, ld, "H");
  if (!rc) rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (alpha < 0 || alpha > 8) return set_error(ACO_ERR_UNSUPPORTED, "alpha must be an integer in [0, 8]");
  if (!(inv_gamma > 0.0f) || !std::isfinite(inv_gamma)) return set_error(ACO_ERR_ARG, "inv_gamma must be > 0");
  return launch_build_P(tau_dev, ACO_FP32, H_dev, n, ld, alpha, inv_gamma, nullptr, nullptr, 1, prec, P_dev,
                        static_cast<cudaStream_t>(stream));
}

int aco_op_construct_shape(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                           int32_t* tours_dev, int32_t* err_dev, int warps, int chunks, int mode,
                           void* stream) {
  int rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m=%d outside [1, %d]", m, ACO_MAX_M);
  if (!tours_dev) return set_error(ACO_ERR_ARG, "tours is NULL");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  rc = prepare_kernels();
  if (rc) return rc;
  ConstructShape s = {warps, chunks, mode};
  return launch_construct(P_dev, prec, n, ld, m, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), it,
                          nullptr, tours_dev, err_dev, s, nullptr, nullptr, nullptr,
                          static_cast<cudaStream_t>(stream));
}

int aco_op_build_lists(const void* P_dev, int prec, int n, int ld, void* lists_dev, int* lcnt_dev,
                       uint32_t* lkey_dev, void* stream) {
  int rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (!lists_dev || !lcnt_dev || !lkey_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (((uintptr_t)lists_dev & 7) != 0) return set_error(ACO_ERR_ARG, "lists must be 8-byte aligned");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  return launch_build_lists(P_dev, prec, n, ld, static_cast<uint2*>(lists_dev), lcnt_dev, lkey_dev,
                            static_cast<cudaStream_t>(stream));
}

int aco_op_build_P_lists(const float* tau_dev, const float* H_dev, int n, int ld, int alpha, float inv_gamma,
                         float rho, int prec, void* P_dev, void* lists_dev, int* lcnt_dev, uint32_t* lkey_dev,
                         void* stream) {
  int rc = check_mat(tau_dev, n, ld, "tau");
  if (!rc) rc = check_mat(H_dev, n, ld, "H");
  if (!rc) rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (!lists_dev || !lcnt_dev || !lkey_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (((uintptr_t)lists_dev & 7) != 0) return set_error(ACO_ERR_ARG, "lists must be 8-byte aligned");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  if (alpha < 0 || alpha > 8) return set_error(ACO_ERR_UNSUPPORTED, "alpha must be an integer in [0, 8]");
  if (!(rho >= 0.0f && rho <= 1.0f)) return set_error(ACO_ERR_ARG, "rho outside [0, 1]");
  return launch_build_P_lists(tau_dev, ACO_FP32, H_dev, n, ld, alpha, inv_gamma, nullptr, nullptr, 1, rho, prec,
                              P_dev, static_cast<uint2*>(lists_dev), lcnt_dev, lkey_dev,
                              static_cast<cudaStream_t>(stream));
}

int aco_op_construct_ex(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                        int32_t* tours_dev, int32_t* err_dev, const void* lists_dev, const int* lcnt_dev,
                        const uint32_t* lkey_dev, int warps, int chunks, int mode, void* stream) {
  int rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m=%d outside [1, %d]", m, ACO_MAX_M);
  if (!tours_dev) return set_error(ACO_ERR_ARG, "tours is NULL");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  if (lists_dev && (!lcnt_dev || !lkey_dev)) return set_error(ACO_ERR_ARG, "lists need lcnt and lkey");
  rc = prepare_kernels();
  if (rc) return rc;
  ConstructShape s = {warps, chunks, mode};
  return launch_construct(P_dev, prec, n, ld, m, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), it,
                          nullptr, tours_dev, err_dev, s, static_cast<const uint2*>(lists_dev), lcnt_dev,
                          lkey_dev, static_cast<cudaStream_t>(stream));
}

int aco_op_construct_rw(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                        int32_t* tours_dev, int32_t* err_dev, void* stream) {
  int rc = check_mat(P_dev, n, ld, "P");
  if (rc) return rc;
  if (m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m=%d outside [1, %d]", m, ACO_MAX_M);
  if (!tours_dev) return set_error(ACO_ERR_ARG, "tours is NULL");
  if (prec < ACO_FP32 || prec > ACO_FP16) return set_error(ACO_ERR_ARG, "unknown precision %d", prec);
  rc = prepare_kernels();
  if (rc) return rc;
  return launch_construct_rw(P_dev, prec, n, ld, m, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), it,
                             nullptr, tours_dev, err_dev, kRwWaitPolls, static_cast<cudaStream_t>(stream));
}

int aco_op_construct(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                     int32_t* tours_dev, int32_t* err_dev, void* stream) {
  return aco_op_construct_shape(P_dev, prec, n, ld, m, seed, it, tours_dev, err_dev, 0, 0, 0, stream);
}

int aco_op_tour_length(const double* D_dev, int n, const int32_t* tours_dev, int m, float Q, double* L_dev,
                       double* c_dev, int32_t* nbr_dev, void* stream) {
  if (!D_dev || !tours_dev || !L_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (n < 3 || n > ACO_MAX_N || m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "n or m out of range");
  if (nbr_dev && ((uintptr_t)nbr_dev & 7)) return set_error(ACO_ERR_ARG, "nbr must be 8-byte aligned");
  const int rc = prepare_kernels();
  if (rc) return rc;
  return launch_tour_length(D_dev, n, tours_dev, m, Q, L_dev, c_dev, nbr_dev, false,
                            static_cast<cudaStream_t>(stream));
}

int aco_op_best(const double* L_dev, const int32_t* tours_dev, int n, int m, int32_t* best_tour_dev,
                double* best_len_dev, void* stream) {
  if (!L_dev || !tours_dev || !best_tour_dev || !best_len_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (n < 3 || n > ACO_MAX_N || m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "n or m out of range");
  return launch_best(L_dev, tours_dev, n, m, best_tour_dev, best_len_dev, nullptr, nullptr, 0, nullptr, nullptr,
                     static_cast<cudaStream_t>(stream));
}

int aco_op_deposit(float* tau_dev, int n, int ld, const int32_t* nbr_dev, const double* c_dev, int m,
                   float rho, int32_t* err_dev, void* stream) {
  int rc = check_mat(tau_dev, n, ld, "tau");
  if (rc) return rc;
  if (!nbr_dev || !c_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m out of range");
  if (!(rho >= 0.0f && rho <= 1.0f)) return set_error(ACO_ERR_ARG, "rho outside [0, 1]");
  rc = prepare_kernels();
  if (rc) return rc;
  return launch_deposit(tau_dev, ACO_FP32, n, ld, nbr_dev, c_dev, m, rho, nullptr, err_dev,
                        static_cast<cudaStream_t>(stream));
}

int aco_op_deposit_atomic(float* tau_dev, int n, int ld, const int32_t* tours_dev, const double* c_dev,
                          int m, float rho, void* stream) {
  int rc = check_mat(tau_dev, n, ld, "tau");
  if (rc) return rc;
  if (!tours_dev || !c_dev) return set_error(ACO_ERR_ARG, "NULL argument");
  if (m < 1 || m > ACO_MAX_M) return set_error(ACO_ERR_ARG, "m out of range");
  if (!(rho >= 0.0f && rho <= 1.0f)) return set_error(ACO_ERR_ARG, "rho outside [0, 1]");
  return launch_deposit_atomic(tau_dev, n, ld, tours_dev, c_dev, m, rho, static_cast<cudaStream_t>(stream));
}

int aco_op_philox(const uint32_t* ctr_dev, uint64_t seed, uint32_t* out_dev, int count, void* stream) {
  if (!ctr_dev || !out_dev || count < 0) return set_error(ACO_ERR_ARG, "invalid argument");
  if (!aligned16(ctr_dev) || !aligned16(out_dev)) return set_error(ACO_ERR_ARG, "buffers must be 16-byte aligned");
  if (count == 0) return ACO_OK;
  return launch_philox(ctr_dev, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), out_dev, count,
                       static_cast<cudaStream_t>(stream));
}

int aco_op_pow_own(const float* x_dev, float e, float* out_dev, int count, void* stream) {
  if (!x_dev || !out_dev || count < 0) return set_error(ACO_ERR_ARG, "invalid argument");
  if (count == 0) return ACO_OK;
  return launch_pow_own(x_dev, e, out_dev, count, static_cast<cudaStream_t>(stream));
}

float aco_gamma(int it, int T, float gamma_max, float gamma_min) { return gamma_at(it, T, gamma_max, gamma_min); }
float aco_inv_gamma(float gamma) { return inv_gamma_of(gamma); }

}  // extern "C"
