/*
 * TensorACO CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, step-by-step C++ restatement of the per-iteration ACO path of
 * "Tensorized Ant Colony Optimization for GPU Acceleration" (Yang, Jiang,
 * Cheng, GECCO'24 Companion):
 *   Sec. 2.1 Eq. 1      transition matrix M_p from M_tau and eta
 *   Sec. 2.2            random start cities T_start, one walk per ant
 *   Sec. 2.4 Eq. 4      independent roulette (IR) and AdaIR selection
 *   Sec. 2.3 Eq. 2/3    index matrix I, increment matrix A, Delta M_tau
 * plus Ant System evaporation tau <- (1-rho) tau (the paper's cited Ant
 * System; the paper itself prints no evaporation formula).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  The GPU library shares no code with it: both sides
 * implement the same published definitions (Philox4x32-10, IEEE rounding,
 * the readings listed below) independently.
 *
 * Readings fixed here (the paper is silent or garbled on them):
 *   - M_p is NOT row-normalised: IR's argmax is invariant to a positive row
 *     scale, so the unnormalised product tau^alpha * eta^beta is used.  FP16
 *     storage alone applies a power-of-two row scale 2^-e_i.
 *   - eta_ij = 1 / max(d_ij, 1e-9); d in fp64 from fp32 coordinates.
 *   - tau^alpha and eta^beta use integer exponents by left-to-right repeated
 *     multiplication (powi), no fused multiply-add anywhere.
 *   - The random deviate r_j of Sec. 2.4 is one uniform per candidate city j,
 *     drawn from Philox4x32-10 with key (seed lo, seed hi) and counter
 *     (j>>2, t, k, it), word j&3, mapped to ((x>>8)|1) * 2^-24 in (0,1).
 *   - T_start holds one start city per ant, in [0,n): Lemire (x*n)>>32 of
 *     word 0 of counter (0, 0, k, it).
 *   - Candidate j replaces the running best iff score > best, or
 *     score == best and j < best_j (lowest index wins ties).
 *   - AdaIR's argmax(r^gamma * p) is computed as argmax(r * p^(1/gamma)):
 *     M_p is raised to 1/gamma once per iteration with pow_own (own log2 /
 *     exp2 polynomials, fp32).  gamma follows a cosine-annealing schedule.
 *   - Evaporation in fp32, the precision of M_tau: tau' = fl32(keep * tau)
 *     with keep = fl32(1 - rho).
 *   - Deposit: every ant deposits c_k = fl64(Q / L_k) on both (i,j) and (j,i)
 *     for each edge of its closed tour; the new tau_ij is tau'_ij plus the
 *     sum of those weights, taken exactly and rounded once to fp32 (the
 *     paper's sum over paths fixes no order, so none is imposed).
 *   - Tour length (Eq. 3): the n fp64 edge lengths of a tour summed exactly
 *     and rounded once to fp64 (the paper's sum fixes no order, so none is
 *     imposed).
 *
 * All matrices here are dense row-major n x n (no padding).
 */
#ifndef TENSORACO_ORACLE_H
#define TENSORACO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FP32 = 0, ORC_BF16 = 1, ORC_FP16 = 2 };

/* ---- random numbers (Philox4x32-10, Salmon et al., SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* word j&3 of Philox(counter=(j>>2, t, k, it), key=seed) */
uint32_t orc_draw(uint64_t seed, uint32_t it, uint32_t k, uint32_t t, uint32_t j);
/* ((x>>8)|1) * 2^-24 : the uniform deviate r in (0,1) of Sec. 2.4 */
float orc_uniform(uint32_t x);
/* T_start entry of ant k at iteration it (Sec. 2.2) */
int32_t orc_start_city(uint64_t seed, uint32_t it, uint32_t k, int32_t n);

/* ---- rounding and elementary functions ---- */
uint16_t orc_to_bf16(float x);
float orc_from_bf16(uint16_t h);
uint16_t orc_to_fp16(float x);
float orc_from_fp16(uint16_t h);
void orc_to_bf16_array(const float* x, uint16_t* out, int64_t count);
void orc_to_fp16_array(const float* x, uint16_t* out, int64_t count);
float orc_powi_f32(float x, int a);
double orc_powi_f64(double x, int a);
float orc_log2_own(float x);
float orc_exp2_own(float y);
float orc_pow_own(float x, float e);
void orc_pow_own_array(const float* x, float e, float* out, int64_t count);
/* cosine-annealed AdaIR gamma for iteration it (Sec. 2.4), rounded to fp32 */
float orc_gamma(int it, int T, float gamma_max, float gamma_min);
/* fl32(1 / gamma) used as the exponent of M_p under AdaIR */
float orc_inv_gamma(float gamma);
/* literal AdaIR deviate r^gamma in fp64 (Eq. 4), for the Eq. 5 law tests */
double orc_adair_deviate(double r, double gamma);

/* ---- Sec. 2.1: distances, heuristic, transition matrix ---- */
void orc_distances(const float* xy, int n, double* D);
void orc_heuristic(const double* D, int n, int beta, float* H);
/* M_p.  P_val receives the value each score multiplies (the stored element
 * widened to fp32); P_bits (nullable) the stored 16-bit pattern for BF16/FP16;
 * row_exp (nullable) the FP16 row exponents e_i. */
void orc_build_P(const float* tau, const float* H, int n, int alpha, float inv_gamma,
                 int prec, float* P_val, uint16_t* P_bits, int32_t* row_exp);

/* ---- Sec. 2.2 / 2.4: tour construction ---- */
/* tours of ants k_begin..k_end-1 into tours[(k-k_begin)*n + t] */
void orc_construct(const float* P_val, int n, uint64_t seed, uint32_t it, int k_begin,
                   int k_end, int32_t* tours, int nthreads);
/* one selection step: argmax over unvisited j of r_j * row[j] (IR) */
int32_t orc_select(const float* row, const uint8_t* visited, int n, uint64_t seed,
                   uint32_t it, uint32_t k, uint32_t t);
/* literal AdaIR step in fp64: argmax over unvisited j of r_j^gamma * row[j] */
int32_t orc_select_literal_adair(const float* row, const uint8_t* visited, int n,
                                 uint64_t seed, uint32_t it, uint32_t k, uint32_t t,
                                 double gamma);

/* Roulette wheel (Sec. 2.4, the selection IR replaces), exact integer
 * reading: q_j = floor(p_j 2^(40-e)), e = floor(log2 max unvisited p); a
 * 64-bit uniform u (Philox counter (2^30, t, k, it), words 0 and 1) picks
 * v = floor(u S / 2^64), S = sum of unvisited q; the first unvisited j whose
 * running sum exceeds v wins (S = 0: the lowest unvisited j). */
uint64_t orc_rw_quantum(float p, int e);
int32_t orc_select_rw(const float* row, const uint8_t* visited, int n, uint64_t seed,
                      uint32_t it, uint32_t k, uint32_t t);
void orc_construct_rw(const float* P_val, int n, uint64_t seed, uint32_t it, int k_begin,
                      int k_end, int32_t* tours, int nthreads);

/* Bernoulli trials of IR on one row q (Sec. 3.3.1): trial tr's deviates
 * come from Philox counter (j>>2, tr lo, tr hi, salt); counts[j] += wins. */
void orc_selection_counts(const float* q, const uint8_t* visited, int n, uint64_t trials,
                          uint64_t seed, uint32_t salt, uint64_t* counts);

/* ---- fitness f (Eq. 3) ---- */
/* L[k] = the exact sum of tour k's n edge lengths D[p_t][p_{t+1 mod n}],
 * rounded once to fp64 (ties to even) */
void orc_tour_lengths(const double* D, int n, const int32_t* tours, int m, double* L);
/* exact sum of count doubles rounded once to fp64 / to fp32 (ties to even) */
double orc_exact_sum(const double* x, int64_t count);
float orc_exact_sum_f32(const double* x, int64_t count);
/* ... rounded once to bfloat16 (returned as its fp32 value); sums >= 0 */
float orc_exact_sum_bf16(const double* x, int64_t count);

/* ---- Sec. 2.3: index matrix, increment matrix, evaporation + deposit ---- */
/* I of one tour (Eq. 2): rows (p_t, p_{t-1}) with cyclic predecessor; out n x 2 */
void orc_index_matrix(const int32_t* tour, int n, int32_t* I);
void orc_deposit(float* tau, int n, const int32_t* tours, const double* L, int m,
                 float rho, float Q);
/* orc_deposit with M_tau stored in bfloat16: the exact sum is rounded once to
 * bf16, untouched entries become bf16(fl32(keep * tau)). */
void orc_deposit_tau_bf16(float* tau, int n, const int32_t* tours, const double* L, int m,
                          float rho, float Q);
/* Sec. 2.3: sort by length (ascending, ties by ant index), select the first
 * k paths (k <= 0 or k >= m: all); deposit from the selected paths only. */
void orc_select_topk(const double* L, int m, int k, uint8_t* selected);
void orc_deposit_topk(float* tau, int n, const int32_t* tours, const double* L, int m,
                      float rho, float Q, int k);
/* float-atomic reading, applied in a caller-given edge order (tests only):
 * tau <- fl32(fl32(1-rho)*tau) then tau[a][b] += fl32(Q/L_k) in fp32 per
 * directed edge, edges visited in the order given by perm (length 2*m*n). */
void orc_deposit_fp32_order(float* tau, int n, const int32_t* tours, const double* L,
                            int m, float rho, float Q, const int64_t* perm);

/* ---- whole iterations ---- */
typedef struct {
  int n, m;
  int alpha, beta;
  float rho, Q;
  uint64_t seed;
  int prec;          /* ORC_FP32 / ORC_BF16 / ORC_FP16 */
  int adair;         /* 0: IR, 1: AdaIR */
  float gamma_max, gamma_min;
  int gamma_T;       /* schedule length */
  int topk;          /* paths that deposit: 0 = all (Ant System), else the k shortest */
  int rw;            /* 1: roulette-wheel construction instead of IR / AdaIR */
  int tau_bf16;      /* 1: M_tau stored in bfloat16 (the run's tau holds bf16 values) */
} orc_params;

/* Runs iterations it0 .. it0+iters-1 in place on tau (n x n) and on the best
 * tour / length (best_len = +inf means none yet).  last_tours (m*n) and
 * last_L (m) receive the final iteration's tours and lengths (nullable). */
void orc_run(const orc_params* prm, const double* D, const float* H, float* tau,
             uint32_t it0, int iters, int32_t* best_tour, double* best_len,
             int32_t* last_tours, double* last_L, int nthreads);
void orc_init_tau(float* tau, int n, float tau0);

#ifdef __cplusplus
}
#endif
#endif
