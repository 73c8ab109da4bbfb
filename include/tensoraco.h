/*
 * tensoraco.h -- C ABI of the GB300 (sm_103a) TensorACO library.
 *
 * The per-iteration path of "Tensorized Ant Colony Optimization for GPU
 * Acceleration" (Yang, Jiang, Cheng, GECCO'24 Companion) for the Euclidean
 * TSP, every step a hand-written CUDA kernel:
 *   (a) M_p = tau^alpha * eta^beta, eta = 1/d               Sec. 2.1, Eq. 1
 *   (b) all m tours by independent roulette (IR) or AdaIR    Sec. 2.2, 2.4, Eq. 4
 *   (c) tour lengths f(s)                                    Eq. 3
 *   (d) evaporate, then deposit Q/f(s) by index mapping      Sec. 2.3, Eq. 2-3
 *
 * Conventions shared by every call:
 *   - Every function returns an int status (ACO_OK = 0, negative on error)
 *     and never aborts; aco_last_error() returns a text for the last error of
 *     the calling thread.
 *   - Sizes are element counts.  n = cities (3 <= n <= ACO_MAX_N),
 *     m = ants (1 <= m <= ACO_MAX_M).  The construction kernels serve
 *     n <= ACO_MAX_N_FP32 with fp32 M_p (ACO_MAX_N_FP32_BATCH in batches),
 *     n <= ACO_MAX_N with bf16 / fp16 M_p, and n <= ACO_MAX_N_RW for the
 *     roulette wheel; solvers and batch instances beyond these are refused
 *     with ACO_ERR_UNSUPPORTED when they are created.
 *   - Arguments named *_host are host pointers, *_dev device pointers.
 *   - Matrices are row-major.  n x n fp32/bf16/fp16 matrices on the device
 *     have a leading dimension `ld` (elements): ld >= n, ld % 8 == 0, base
 *     address 16-byte aligned.  Padding columns j >= n are never read as
 *     candidates.  Distance matrices are fp64 n x n with leading dimension n.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device-
 *     pointer calls are asynchronous on that stream; host-pointer calls
 *     synchronise it before returning.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed
 *     (low word, high word), counter (j>>2, t, k, it), word j&3 for candidate
 *     j at step t of ant k in iteration it; deviate ((x>>8)|1) * 2^-24.
 *     Start city of ant k: (x*n)>>32, x = word 0 of counter (0, 0, k, it).
 *   - alpha and beta must be integers in [0, 8] (integer powers by repeated
 *     multiplication keep every result reproducible bit for bit).
 */
#ifndef TENSORACO_H
#define TENSORACO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ACO_OK 0
#define ACO_ERR_ARG (-1)         /* invalid argument */
#define ACO_ERR_OOM (-2)         /* device allocation failed / workspace too small */
#define ACO_ERR_CUDA (-3)        /* a CUDA runtime call or kernel failed */
#define ACO_ERR_STATE (-4)       /* call out of order (e.g. best before any iteration) */
#define ACO_ERR_UNSUPPORTED (-5) /* valid request this build does not support */
#define ACO_ERR_TIMEOUT (-6)     /* a bounded device-side wait ran out */

#define ACO_MAX_N 65536
#define ACO_MAX_N_FP32 49152       /* fp32 M_p: a row staged in at most 192 KB of shared memory */
#define ACO_MAX_N_FP32_BATCH 32768 /* fp32 M_p inside batches */
#define ACO_MAX_N_RW 16384         /* roulette-wheel construction */
#define ACO_MAX_M 1048576

enum { ACO_FP32 = 0, ACO_BF16 = 1, ACO_FP16 = 2 };           /* storage of M_p */
enum { ACO_IR = 0, ACO_ADAIR = 1, ACO_RW = 2 };               /* selection, Sec. 2.4 */
enum { ACO_DEPOSIT_DET = 0, ACO_DEPOSIT_ATOMIC = 1 };        /* Delta M_tau summation */

/* Text of the calling thread's last error ("" if none). Never NULL. */
const char* aco_last_error(void);

/* ======================================================================
 * Single-instance API.  One global solver, not thread-safe; the handle API
 * below gives independent solvers.
 * ==================================================================== */

/* Create the global solver on the current device: copies coords_host
 * (n x 2 fp32, (x, y) per city) to the device, builds the fp64 distance
 * matrix and eta^beta, sets tau = 1 (Sec. 2.1).  rho in [0,1], Q > 0,
 * alpha/beta integers in [0,8].  Replaces a previous global solver.
 * Uses the workspace given to aco_bind() when one is bound, else allocates. */
int aco_init(const float* coords_host, int n, int m, float alpha, float beta, float rho,
             float Q, uint64_t seed);

/* Selection mechanism (Sec. 2.4).  ACO_RW is the roulette wheel IR replaces,
 * in an exact integer reading: with e = floor(log2 max unvisited p),
 * q_j = floor(p_j 2^(40-e)), S the sum of the unvisited q, a 64-bit uniform u
 * from Philox counter (2^30, t, k, it) (words 0, 1) and v = floor(u S / 2^64),
 * the next city is the first unvisited j whose running sum of q exceeds v
 * (S = 0: the lowest unvisited j); n <= 16384, no candidate lists.  ACO_IR
 * ignores the gammas.  ACO_ADAIR
 * anneals gamma from gamma_max to gamma_min over T iterations by a cosine
 * schedule (gamma_t = gmin + (gmax-gmin)/2 (1 + cos(pi t / T)), gmin after T)
 * and selects argmax(r^gamma p) in the equivalent form argmax(r p^(1/gamma)).
 * gamma_* in (0, 16], T >= 1.  Takes effect at the next iteration. */
int aco_set_variant(int roulette, float gamma_max, float gamma_min, int T);

/* Storage precision of M_p: ACO_FP32, ACO_BF16 (RNE), ACO_FP16 (RNE after a
 * per-row power-of-two scale 2^-e_i placing the row maximum in [2^14, 2^15)).
 * Scores are always fp32; tau is stored as aco_set_tau_precision selects.
 * Takes effect at the next iteration. */
int aco_set_precision(int prec);

/* Storage precision of M_tau: ACO_FP32 (default) or ACO_BF16.  With BF16 the
 * deposit rounds fl32(keep * tau) + the exact sum of the weights once to bf16
 * (entries no path uses: bf16(fl32(keep * tau))), tau starts at bf16(tau0),
 * M_p widens it exactly.  Needs ACO_DEPOSIT_DET.  Next aco_init. */
int aco_set_tau_precision(int prec);

/* Deposit summation: ACO_DEPOSIT_DET gives every entry the exact sum of its
 * paths' weights added to the evaporated value, rounded once to fp32 (no
 * order; reproducible bit for bit); ACO_DEPOSIT_ATOMIC adds fl32(Q/L_k) with
 * fp32 atomics in hardware order (not reproducible). */
int aco_set_deposit(int mode);

/* Deposit path selection (Sec. 2.3: the solution set is sorted by fitness
 * and the top k paths deposit; the paper's experiments use k = n/10): the
 * k >= 1 shortest tours of each iteration deposit (equal lengths: lower ant
 * index first), every entry still evaporates; k = 0 (default) or k >= m:
 * every ant deposits.  Takes effect at the next iteration. */
int aco_set_deposit_topk(int k);

/* Run k >= 0 iterations (a)-(d).  Iterations are numbered from 0 across calls.
 * Asynchronous on the bound stream. */
int aco_iterate(int k);

/* Best tour so far (n city indices into tour_host) and its length.  The best
 * is replaced only by a strictly shorter tour; within an iteration the lowest
 * ant index wins ties.  ACO_ERR_STATE before the first iteration. */
int aco_best(int32_t* tour_host, double* len_host);

/* Copies of the current state to host memory: tau (n x n, dense),
 * last iteration's tours (m x n) and lengths (m). */
int aco_get_tau(float* tau_host);
int aco_get_tours(int32_t* tours_host);
int aco_get_lengths(double* lengths_host);

/* Release the global solver (and its workspace if the library allocated it). */
int aco_free(void);

/* Device bytes one solver of (n, m) needs, whatever the precision. */
int aco_workspace_bytes(int n, int m, int prec, size_t* bytes);

/* Give the next aco_init a caller-owned device workspace (e.g. a torch
 * tensor) of `bytes` >= aco_workspace_bytes(), 256-byte aligned, and the
 * stream all its work is issued on.  The caller keeps ownership and must keep
 * the memory alive until aco_free().  dev_workspace NULL unbinds.  stream
 * NULL: the library's own stream, created once per process with default
 * flags (so ordered with the legacy default stream both ways), on which an
 * iteration is replayed as one CUDA graph. */
int aco_bind(void* dev_workspace, size_t bytes, void* stream);

/* ======================================================================
 * Handle API: independent solvers (used by the batch and serving layers).
 * ==================================================================== */
typedef struct aco_solver aco_solver;

typedef struct {
  int n, m;
  int alpha, beta;          /* integers in [0, 8] */
  float rho, Q, tau0;       /* rho in [0,1], Q > 0, tau0 > 0 */
  uint64_t seed;
  int prec;                 /* ACO_FP32 / ACO_BF16 / ACO_FP16 */
  int roulette;             /* ACO_IR / ACO_ADAIR / ACO_RW */
  int deposit;              /* ACO_DEPOSIT_DET / ACO_DEPOSIT_ATOMIC */
  float gamma_max, gamma_min;
  int gamma_T;
  int cand_lists;           /* 1: candidate-list fast path (exact), 0: full scan only */
  int topk;                 /* paths that deposit (Sec. 2.3): 0 = all (Ant System), else the
                               topk shortest (ties: lower ant index); >= m means all */
  int tau_prec;             /* storage of M_tau: ACO_FP32 (default) or ACO_BF16 (deterministic
                               deposit only) */
} aco_params;

/* Fill *p with defaults: alpha 1, beta 2, rho 0.5, Q 1, tau0 1, seed 0, FP32,
 * IR, deterministic deposit, gamma 1.5 -> 0.5 over 100 iterations, candidate
 * lists on. */
int aco_params_default(aco_params* p);

/* Create a solver for p->n cities given coords_host (n x 2 fp32).  Workspace:
 * dev_workspace/ws_bytes as for aco_bind (NULL: the library allocates).
 * stream: the solver's stream (NULL: legacy default stream). */
int aco_create(aco_solver** out, const float* coords_host, const aco_params* p,
               void* dev_workspace, size_t ws_bytes, void* stream);
int aco_destroy(aco_solver* s);
int aco_solver_iterate(aco_solver* s, int k);
int aco_solver_best(aco_solver* s, int32_t* tour_host, double* len_host);
int aco_solver_get_tau(aco_solver* s, float* tau_host);
int aco_solver_get_tours(aco_solver* s, int32_t* tours_host);
int aco_solver_get_lengths(aco_solver* s, double* lengths_host);
/* Device pointers into the solver's state (borrowed, valid until destroy):
 * tau (leading dimension *ld; fp32, or bf16 bit patterns when the solver
 * stores M_tau in bf16), tours (int32 m x n), lengths (fp64 m), best tour
 * (int32 n), best length (fp64 1). */
int aco_solver_device_state(aco_solver* s, float** tau, int* ld, int32_t** tours,
                            double** lengths, int32_t** best_tour, double** best_len);
/* Iterations completed so far. */
int aco_solver_iteration(aco_solver* s, uint32_t* it);

/* Checkpoints.  A solver's state -- tau, the best tour and length, the
 * iteration count, and its parameters -- as a host byte blob of
 * aco_solver_state_bytes() bytes, ending in an FNV-1a 64-bit checksum.
 * Everything else is derived (M_p and lists from tau, distances from the
 * coordinates, random numbers from seed and counters), so a solver restored
 * into one created with the same coordinates and parameters continues bit
 * for bit as the saved one would.  aco_solver_load returns ACO_ERR_ARG for a
 * blob of another size, format, checksum or parameter set; the solver is then
 * unchanged.  Both synchronise the solver's stream. */
int aco_solver_state_bytes(aco_solver* s, size_t* bytes);
int aco_solver_save(aco_solver* s, void* host_buf, size_t bytes);
int aco_solver_load(aco_solver* s, const void* host_buf, size_t bytes);

/* Kernel timing probes.  When on, the solver records CUDA events around each
 * kernel of every iteration (inside its CUDA graph as well).  After an
 * iteration has been issued, aco_solver_kernel_ms() waits for it and writes
 * the durations in milliseconds of its six steps, in order: build_P,
 * build_lists (0 without candidate lists), construct, tour_length, best,
 * deposit (evaporation + deposit for the atomic mode). */
int aco_solver_set_profiling(aco_solver* s, int on);
int aco_solver_kernel_ms(aco_solver* s, float* ms6);

/* Bound on each roulette-wheel step's wait for the copy of its row of M_p
 * (ACO_RW solvers), in polls of the copy's mbarrier; the default,
 * ACO_WAIT_POLLS_DEFAULT, is far above a normal copy's wait.  A wait that
 * runs out makes that ant's CTA record it, let the copy land and stop; the
 * next call that synchronises the solver returns ACO_ERR_TIMEOUT, once (the
 * solver's error word is cleared when read).  That iteration's tours and the
 * state it updated are not meaningful: restore a checkpoint.  polls = 0 makes
 * every wait give up at once, which exercises this path.  Takes effect at
 * the next iteration. */
#define ACO_WAIT_POLLS_DEFAULT 1048576u
int aco_solver_set_wait_polls(aco_solver* s, uint32_t polls);

/* Choose the construct launch shape (warps, chunks, mode as for
 * aco_op_construct_shape) for this solver: warps = chunks = 0 restores the
 * default (autotuned if aco_autotune_construct ran for its n, m and precision). */
int aco_solver_set_shape(aco_solver* s, int warps, int chunks, int mode);

/* ======================================================================
 * Batches: many independent instances advanced together.  One iteration of
 * a batch is a few multi-instance launches over all active instances -- one
 * CTA per (instance, row) for M_p, the candidate lists and the deposit, one
 * persistent launch for the construction of every ant of every IR / AdaIR
 * instance (work items handed out by a global counter, largest n first), one
 * CTA per ant of the roulette-wheel instances, one warp per (instance, ant)
 * for the lengths, one CTA per instance for the best -- replayed as a CUDA
 * graph while the active set is unchanged.  Each instance keeps its whole state
 * (tau, M_p, tours, best) resident in a workspace carved from the batch's
 * device arena by a first-fit allocator; results are bit-identical to those
 * of a single solver with the same parameters.
 * ==================================================================== */
typedef struct aco_batch aco_batch;

/* max_instances: slot table size.  arena_bytes: device memory for instance
 * workspaces; dev_arena (256-byte aligned, caller-owned, nullable) provides
 * it, else the library allocates it.  All instances share `prec`.  stream:
 * the batch's stream (NULL: legacy default stream, no graph replay). */
int aco_batch_create(aco_batch** out, int max_instances, size_t arena_bytes, int prec,
                     void* dev_arena, void* stream);
int aco_batch_destroy(aco_batch* b);

/* Admit an instance: coords_host n x 2 fp32, p as for aco_create (p->prec
 * must equal the batch's; p->tau_prec and p->roulette may differ between
 * instances: roulette-wheel instances (Sec. 2.4, n <= 16384) are built by
 * their own multi-instance kernel, one CTA per ant).  It runs
 * iters_budget iterations (0: until removed), then stops advancing and
 * keeps its results.  *slot receives its slot id.  ACO_ERR_OOM (nothing
 * changed) when no slot is free or its workspace (aco_batch_instance_bytes)
 * does not fit in the arena now. */
int aco_batch_add(aco_batch* b, const float* coords_host, const aco_params* p, int iters_budget,
                  int* slot);
/* Release a slot and its workspace. */
int aco_batch_remove(aco_batch* b, int slot);
/* Run k iterations of every active (unfinished) instance. */
int aco_batch_step(aco_batch* b, int k);
int aco_batch_best(aco_batch* b, int slot, int32_t* tour_host, double* len_host);
/* M_tau of a slot as n x n fp32 (bf16 storage widened exactly). */
int aco_batch_get_tau(aco_batch* b, int slot, float* tau_host);
int aco_batch_status(aco_batch* b, int slot, uint32_t* iterations_done, int* finished);
/* Active instances, free arena bytes and largest free block. */
int aco_batch_info(aco_batch* b, int* active, size_t* free_bytes, size_t* largest_block);
/* Construct launch shape for the batch (0, 0, 0: the default covering the
 * largest active n). */
int aco_batch_set_shape(aco_batch* b, int warps, int chunks, int mode);
/* Arena bytes one instance of (n, m) takes. */
int aco_batch_instance_bytes(int n, int m, size_t* bytes);

/* ======================================================================
 * Step-level API on caller-owned device buffers (one kernel family each),
 * asynchronous on `stream`.  The solvers above are built from these.
 * ==================================================================== */

/* Sec. 2.1: D_ij = sqrt(dx^2 + dy^2) in fp64 (D_dev n x n, nullable) and
 * H_ij = fl32(powi_f64(1 / max(D_ij, 1e-9), beta)), H_ii = 0 (H_dev n x ld),
 * from coords_dev (n x 2 fp32). */
int aco_op_heuristic(const float* coords_dev, int n, int beta, double* D_dev, float* H_dev,
                     int ld, void* stream);

/* Fill an n x ld fp32 matrix with `value` (tau initialisation). */
int aco_op_fill(float* dev, int n, int ld, float value, void* stream);

/* Eq. 1 (unnormalised): X_ij = fl32(powi_f32(tau_ij, alpha) * H_ij), X_ii = 0;
 * AdaIR (inv_gamma != 1): X_ij <- pow_own(X_ij, inv_gamma); then stored at
 * `prec` into P_dev (n x ld; 4 bytes per element for ACO_FP32, 2 otherwise).
 * Padding columns are written as 0. */
int aco_op_build_P(const float* tau_dev, const float* H_dev, int n, int ld, int alpha,
                   float inv_gamma, int prec, void* P_dev, void* stream);

/* Sec. 2.2 + 2.4: tours of ants 0..m-1 at iteration `it` over M_p (P_dev,
 * n x ld at `prec`) into tours_dev (m x n int32).  Each step selects
 * argmax over unvisited j of fl32(r_j * P[cur, j]), lowest j on ties.
 * err_dev (nullable, int32) is set non-zero if a kernel-side check failed. */
int aco_op_construct(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed,
                     uint32_t it, int32_t* tours_dev, int32_t* err_dev, void* stream);

/* Same, with an explicit launch shape: warps per ant, 16-byte chunks per
 * lane (32*warps*chunks*(16/elem bytes) >= n) and mode (0: the row is staged
 * in shared memory by cp.async, 1: direct register loads).  warps = 0 picks
 * the default.  ACO_ERR_UNSUPPORTED when the shape is not compiled in. */
int aco_op_construct_shape(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed,
                           uint32_t it, int32_t* tours_dev, int32_t* err_dev, int warps,
                           int chunks, int mode, void* stream);

/* Candidate lists of M_p, the exact fast path of the construction step: for
 * each row i, lcnt_dev[i] <= ACO_LIST_MAX entries lists_dev[i*ACO_LIST_MAX + q]
 * = (fp32 bits of the stored value, column), sorted by value (descending,
 * ties by column) -- every column whose value is above the row's
 * ACO_LIST_TARGET-th largest value T, then columns equal to T in column order
 * while room remains (every column when n <= ACO_LIST_MAX) -- and
 * lkey_dev[i] bounds the score key (fp32 bits + 1) of every column not
 * listed: T when all columns >= T are listed, T + 1 when ties at T were cut,
 * 0 when nothing is left out.  lists_dev: n*ACO_LIST_MAX pairs of u32,
 * 8-byte aligned; lcnt_dev, lkey_dev: n entries. */
#define ACO_LIST_TARGET 256
#define ACO_LIST_MAX 512
int aco_op_build_lists(const void* P_dev, int prec, int n, int ld, void* lists_dev, int* lcnt_dev,
                       uint32_t* lkey_dev, void* stream);

/* aco_op_build_P and aco_op_build_lists in one pass (the solvers' and
 * batches' form): the same M_p, lists, counts and bounds.  lkey_dev also
 * serves as input: each row's previous bound, scaled by the evaporation
 * (1 - rho)^alpha, is the threshold above which the pass collects candidates;
 * when that collects between ACO_LIST_TARGET and ACO_LIST_MAX columns the
 * list is sorted from them, otherwise it is selected from the whole row as
 * aco_op_build_lists does.  Any lkey_dev contents give the same results; only
 * the time depends on them.  tau_dev fp32. */
int aco_op_build_P_lists(const float* tau_dev, const float* H_dev, int n, int ld, int alpha, float inv_gamma,
                         float rho, int prec, void* P_dev, void* lists_dev, int* lcnt_dev, uint32_t* lkey_dev,
                         void* stream);

/* Sec. 2.4 roulette wheel (ACO_RW above) for all m ants on M_p; n <= 16384
 * (ACO_ERR_UNSUPPORTED beyond).  Arguments as for aco_op_construct. */
int aco_op_construct_rw(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                        int32_t* tours_dev, int32_t* err_dev, void* stream);

/* aco_op_construct_shape with candidate lists (from aco_op_build_lists on the
 * same M_p; lists_dev NULL: full scan only).  The tours are the same either
 * way: a step is taken from the list only when no unlisted column can win. */
int aco_op_construct_ex(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed,
                        uint32_t it, int32_t* tours_dev, int32_t* err_dev, const void* lists_dev,
                        const int* lcnt_dev, const uint32_t* lkey_dev, int warps, int chunks,
                        int mode, void* stream);

/* Eq. 3 and the index mapping of Eq. 2: L_k = sum_t D[p_t][p_{t+1 mod n}],
 * the exact sum of the n fp64 edge lengths rounded once to fp64 (ties to
 * even; Eq. 3 fixes no order, so the result depends on none) (L_dev, m),
 * c_k = fl64(Q / L_k) (c_dev, m), and for every city a the neighbours of a in
 * tour k: nbr_dev[(a*m + k)*2 + {0,1}] = (predecessor, successor) (nbr_dev:
 * n*m*2 int32, nullable).  The exact sum holds edge lengths of 0 or in
 * [2^-149, 2^130) -- every distance of fp32 coordinates; a tour with any
 * other edge length gets L_k = c_k = NaN.  Tours are permutations of 0..n-1;
 * for a city some tour misses, that ant's nbr entry is -1 or left as it was
 * (entries outside [0, n) are skipped by the deposit). */
int aco_op_tour_length(const double* D_dev, int n, const int32_t* tours_dev, int m, float Q,
                       double* L_dev, double* c_dev, int32_t* nbr_dev, void* stream);

/* Iteration best (argmin L, lowest k on ties) merged into the running best:
 * replaced only if strictly shorter.  best_len_dev starts at +inf. */
int aco_op_best(const double* L_dev, const int32_t* tours_dev, int n, int m,
                int32_t* best_tour_dev, double* best_len_dev, void* stream);

/* Sec. 2.3, deterministic: tau'_ab = fl32(keep * tau_ab), keep = fl32(1 - rho)
 * (fp32); an entry (a,b) on the tour of some ant becomes tau'_ab plus the
 * c_k of every such ant, summed exactly and rounded once to fp32 (ties to
 * even); other entries become tau'_ab.  The sum is exact, so no order of the
 * ants is involved.  Input: nbr/c from aco_op_tour_length; every c_k must be
 * >= 0 or +inf (+inf makes the entries of that tour +inf) and the positive
 * finite ones must lie within a factor 2^19 of each other (true for the
 * tour lengths of one planar instance).  Otherwise every entry some path
 * uses becomes NaN, the others tau'_ab, and *err_dev (nullable, device
 * int32) is set to 2.  tau_dev n x ld, 16-byte aligned, updated in place. */
int aco_op_deposit(float* tau_dev, int n, int ld, const int32_t* nbr_dev, const double* c_dev,
                   int m, float rho, int32_t* err_dev, void* stream);

/* Selection frequencies of independent roulette on one row (the Bernoulli
 * trials of the paper's AdaIR visualisation, Sec. 3.3.1): for each of
 * `trials` trials, r_j from Philox4x32-10 with key seed and counter
 * (j >> 2, tr mod 2^32, tr div 2^32, salt), word j & 3, mapped as in the
 * construction; the unvisited j maximising fl32(r_j * q_dev[j]) (lowest j on
 * ties) gets counts_dev[j] += 1.  q_dev: n fp32 (for AdaIR the row raised to
 * 1/gamma); visited_dev: n bytes, nonzero = excluded (nullable); counts_dev:
 * n u64, accumulated into (zero it first).  n <= 4096. */
int aco_op_selection_counts(const float* q_dev, const uint8_t* visited_dev, int n,
                            unsigned long long trials, uint64_t seed, uint32_t salt,
                            unsigned long long* counts_dev, void* stream);

/* Sec. 2.3 path selection: with the lengths L_dev (m fp64) sorted ascending
 * (equal lengths by ant index), set c_dev[j] = 0 for every ant j outside the
 * first k, so that aco_op_deposit deposits from the k shortest paths only.
 * k <= 0 or k >= m: c_dev is left unchanged.  One CTA; device buffers. */
int aco_op_select_topk(const double* L_dev, int m, int k, double* c_dev, void* stream);

/* Sec. 2.3, float-atomic: tau <- fl32(fl32(1-rho) tau), then for every
 * directed tour edge (a,b) of ant k: atomicAdd(tau_ab, fl32(c_k)). */
int aco_op_deposit_atomic(float* tau_dev, int n, int ld, const int32_t* tours_dev,
                          const double* c_dev, int m, float rho, void* stream);

/* Allocation-free tour lengths + deterministic deposit.  The paper has no
 * counterpart.  It serves callers that cannot allocate device memory where
 * they update the pheromone: embedders whose device memory all belongs to a
 * framework pool or a budget fixed at start-up, and loops with a latency
 * bound, where a cudaMalloc (which may synchronise the device and has no
 * bounded running time) is not allowed.
 * Same results as aco_op_tour_length(D_dev, n, tours_dev, m, Q, L_dev, c, nbr)
 * followed by aco_op_deposit(tau_dev, n, ld, nbr, c, m, rho, err_dev), but the
 * scratch c (m fp64) and nbr (2*n*m int32) lives in a fixed device array
 * inside the library of ACO_NOALLOC_SCRATCH_BYTES (16 MiB; every GPU that
 * loads the library holds it until exit), so 8*m (rounded up to 256) + 8*n*m
 * must fit: larger n*m returns ACO_ERR_ARG before any device work.
 * Inputs/outputs as for the two calls above; L_dev (m fp64) receives the
 * lengths, tau_dev is updated in place, *err_dev (nullable, device int32) is
 * set to 2 when the weights Q / L_k cannot be summed exactly (the touched
 * entries are then NaN).  Allocates nothing.  Its first call on a device
 * looks up the array's device address with cudaGetSymbolAddress; make that
 * first call before any stream capture.  Every call clears the array's
 * index mapping before use.  All calls share the array: calls that overlap
 * on the GPU race. */
#define ACO_NOALLOC_SCRATCH_BYTES (16u << 20)
int aco_op_deposit_tours_noalloc(float* tau_dev, int n, int ld, const double* D_dev,
                                 const int32_t* tours_dev, int m, float rho, float Q,
                                 double* L_dev, int32_t* err_dev, void* stream);

/* Autotuner: times every compiled construct shape that covers n on the
 * given M_p (reps launches each, after one warm-up) and registers the fastest
 * as the default for (n, m, prec) in this process.  tours_scratch_dev: m x n
 * int32.  Outputs the chosen shape and its mean time in ms (nullable). */
int aco_autotune_construct(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed,
                           int32_t* tours_scratch_dev, int reps, int* warps_out, int* chunks_out,
                           int* mode_out, float* ms_out, void* stream);

/* Test utilities: Philox4x32-10 blocks for count counters (ctr_dev 4*count
 * u32, out_dev 4*count u32) under key (seed lo, hi); and the device pow_own
 * used by AdaIR on count fp32 values. */
int aco_op_philox(const uint32_t* ctr_dev, uint64_t seed, uint32_t* out_dev, int count,
                  void* stream);
int aco_op_pow_own(const float* x_dev, float e, float* out_dev, int count, void* stream);

/* Construction with step probes (a measurement utility; the paper has no
 * counterpart): aco_op_construct_ex's candidate-list construction of all m
 * ants (same tours; 32 <= n <= 16384, lists from aco_op_build_lists) in which
 * ant probe_ant also records each step t = 1..n-1 as 8 u32 at
 * probe_dev[8*t ..]: the SM clock at the step's start; the cycles from it
 * until the step's first list entry is available, its Philox block is done,
 * its speculative list loads are issued, the first round's decision, the
 * decision after any slower path, and the end of the step; flags (1: the
 * first round decided, 2: later list rounds ran, 4: a full scan ran, 8 / 16:
 * the next list came from speculation slot 0 / 1).  probe_dev: 8*n u32.  The
 * clock reads cost a few cycles of their own. */
int aco_op_construct_probe(const void* P_dev, int prec, int n, int ld, int m, uint64_t seed, uint32_t it,
                           int32_t* tours_dev, int32_t* err_dev, const void* lists_dev, const uint32_t* lkey_dev,
                           int probe_ant, uint32_t* probe_dev, void* stream);

/* Roofline ceilings of the construction step (measurement utilities; the
 * paper has no counterpart).  Each launch is asynchronous on `stream`; time it
 * with events and divide the work it states by the time.  sink_dev: one
 * device u64 the kernels add a checksum to (keeps their work observable).
 *   aco_ceiling_row_reads: `warps` warps (a multiple of 8) each read
 *     rows_per_warp whole rows, chosen at random (salt varies the choice), of
 *     a buffer of `bytes` bytes cut into rows of row_bytes (a multiple of 16)
 *     with 16-byte coalesced loads -- the full-scan construction's reads of
 *     M_p rows (Sec. 2.4).  Work: warps * rows_per_warp * row_bytes bytes.
 *   aco_ceiling_philox: `threads` threads (a multiple of 256) each draw
 *     blocks_per_thread Philox4x32-10 blocks and score their four words as
 *     candidates (fl32(r * p), running argmax) -- a step's arithmetic per
 *     candidate.  Work: 4 * threads * blocks_per_thread candidates.
 *   aco_ceiling_chase: `chains` CTAs each follow `hops` dependent loads
 *     j <- next_dev[j] (next_dev: a permutation of 0..slots-1, u32) from slot
 *     977 * chain; cycles_dev[chain] (u64) receives clock cycles per load. */
int aco_ceiling_row_reads(const void* buf_dev, size_t bytes, int row_bytes, int warps, int rows_per_warp,
                          uint32_t salt, unsigned long long* sink_dev, void* stream);
int aco_ceiling_philox(uint64_t seed, int threads, int blocks_per_thread, uint32_t salt,
                       unsigned long long* sink_dev, void* stream);
int aco_ceiling_chase(const uint32_t* next_dev, size_t slots, int chains, int hops,
                      unsigned long long* cycles_dev, unsigned long long* sink_dev, void* stream);

/* Cosine-annealed gamma of iteration it (host, fp64 rounded to fp32) and
 * fl32(1/gamma); the same values the solvers use. */
float aco_gamma(int it, int T, float gamma_max, float gamma_min);
float aco_inv_gamma(float gamma);

#ifdef __cplusplus
}
#endif
#endif /* TENSORACO_H */
