// TensorACO CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// The per-iteration ACO path, step by step, in the paper's order:
//   Sec. 2.1 (Eq. 1)  M_p from M_tau^alpha and eta^beta
//   Sec. 2.2          T_start, then each ant walks n-1 steps
//   Sec. 2.4          each step: v = argmax(r (.) p_u) over unvisited cities
//   Eq. 3             fitness f = closed tour length
//   Sec. 2.3 (Eq. 2/3) index matrix I, increment A, Delta M_tau = sum of A
// plus Ant System evaporation before the deposit.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

extern "C" {

// d_ij = sqrt(dx^2 + dy^2) in fp64 from fp32 coordinates (x_i, y_i) = xy[2i], xy[2i+1].
void orc_distances(const float* xy, int n, double* D) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double dx = (double)xy[2 * i] - (double)xy[2 * j];
      double dy = (double)xy[2 * i + 1] - (double)xy[2 * j + 1];
      D[(size_t)i * n + j] = std::sqrt(dx * dx + dy * dy);
    }
  }
}

// eta^beta (Sec. 2.1): eta_ij = 1 / max(d_ij, 1e-9), raised to the integer beta
// in fp64, rounded once to fp32.  The diagonal is never a candidate: 0.
void orc_heuristic(const double* D, int n, int beta, float* H) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      if (i == j) {
        H[(size_t)i * n + j] = 0.0f;
        continue;
      }
      double d = D[(size_t)i * n + j];
      double eta = 1.0 / (d > 1e-9 ? d : 1e-9);
      H[(size_t)i * n + j] = (float)orc_powi_f64(eta, beta);
    }
  }
}

// M_p (Eq. 1) without row normalisation: X_ij = fl32(tau_ij^alpha * eta_ij^beta);
// under AdaIR X_ij <- X_ij^(1/gamma); then stored at the chosen precision.
// FP16 storage divides row i by 2^e_i, e_i = clamp(floor(log2(max_j X_ij)) - 14,
// -126, 113) (0 for an all-zero row), so that the row maximum lies in [2^14, 2^15).
void orc_build_P(const float* tau, const float* H, int n, int alpha, float inv_gamma,
                 int prec, float* P_val, uint16_t* P_bits, int32_t* row_exp) {
  std::vector<float> X((size_t)n);
  for (int i = 0; i < n; ++i) {
    float rowmax = 0.0f;
    for (int j = 0; j < n; ++j) {
      float x = 0.0f;
      if (j != i) {
        x = orc_powi_f32(tau[(size_t)i * n + j], alpha) * H[(size_t)i * n + j];
        if (inv_gamma != 1.0f) x = orc_pow_own(x, inv_gamma);
      }
      X[j] = x;
      if (x > rowmax) rowmax = x;
    }
    int e = 0;
    if (prec == ORC_FP16 && rowmax > 0.0f) {
      uint32_t b;
      std::memcpy(&b, &rowmax, 4);
      int ef = (int)((b >> 23) & 0xFF);
      int fl2 = (ef == 0) ? -127 : ef - 127;
      e = fl2 - 14;
      if (e < -126) e = -126;
      if (e > 113) e = 113;
    }
    if (row_exp) row_exp[i] = e;
    // 2^-e as an exact fp32 power of two (-e in [-113, 126])
    uint32_t sb = (uint32_t)(127 - e) << 23;
    float scale;
    std::memcpy(&scale, &sb, 4);
    for (int j = 0; j < n; ++j) {
      size_t idx = (size_t)i * n + j;
      if (prec == ORC_FP32) {
        P_val[idx] = X[j];
        if (P_bits) P_bits[idx] = 0;
      } else if (prec == ORC_BF16) {
        uint16_t h = orc_to_bf16(X[j]);
        P_val[idx] = orc_from_bf16(h);
        if (P_bits) P_bits[idx] = h;
      } else {
        uint16_t h = orc_to_fp16(X[j] * scale);
        P_val[idx] = orc_from_fp16(h);
        if (P_bits) P_bits[idx] = h;
      }
    }
  }
}

// One IR selection (Sec. 2.4): v = argmax over unvisited j of r_j * p_j with
// r_j the Philox deviate of (it, k, t, j).  Ties go to the lowest j.
int32_t orc_select(const float* row, const uint8_t* visited, int n, uint64_t seed,
                   uint32_t it, uint32_t k, uint32_t t) {
  int32_t best_j = -1;
  float best = 0.0f;
  for (int j = 0; j < n; ++j) {
    if (visited[j]) continue;
    float r = orc_uniform(orc_draw(seed, it, k, t, (uint32_t)j));
    float score = r * row[j];
    if (best_j < 0 || score > best || (score == best && j < best_j)) {
      best = score;
      best_j = j;
    }
  }
  return best_j;
}

// The literal AdaIR step of Eq. 4 in fp64: argmax over unvisited j of r_j^gamma * p_j.
int32_t orc_select_literal_adair(const float* row, const uint8_t* visited, int n,
                                 uint64_t seed, uint32_t it, uint32_t k, uint32_t t,
                                 double gamma) {
  int32_t best_j = -1;
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    if (visited[j]) continue;
    double r = (double)orc_uniform(orc_draw(seed, it, k, t, (uint32_t)j));
    double score = std::pow(r, gamma) * (double)row[j];
    if (best_j < 0 || score > best || (score == best && j < best_j)) {
      best = score;
      best_j = j;
    }
  }
  return best_j;
}

// Sec. 2.2: ant k starts at T_start[k] and takes n-1 IR steps over M_p.
static void construct_one(const float* P_val, int n, uint64_t seed, uint32_t it, int k,
                          int32_t* tour) {
  std::vector<uint8_t> visited((size_t)n, 0);
  int32_t cur = orc_start_city(seed, it, (uint32_t)k, n);
  tour[0] = cur;
  visited[cur] = 1;
  for (int t = 1; t < n; ++t) {
    int32_t v = orc_select(P_val + (size_t)cur * n, visited.data(), n, seed, it,
                           (uint32_t)k, (uint32_t)t);
    tour[t] = v;
    visited[v] = 1;
    cur = v;
  }
}

void orc_construct(const float* P_val, int n, uint64_t seed, uint32_t it, int k_begin,
                   int k_end, int32_t* tours, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int k = k_begin; k < k_end; ++k)
    construct_one(P_val, n, seed, it, k, tours + (size_t)(k - k_begin) * n);
  (void)nthreads;
}

// ---------------------------------------------------------------------------
// Roulette wheel (Sec. 2.4: the classical selection that IR replaces): the
// next city is drawn with probability proportional to p_j over the unvisited
// j.  Exact integer reading, so that every summation order agrees:
//   e    = floor(log2 of the largest unvisited p_j)
//   q_j  = floor(p_j * 2^(40 - e))        (the largest q lies in [2^40, 2^41))
//   S    = sum of q_j over the unvisited j
//   u    = words 0 (high) and 1 (low) of Philox(counter (2^30, t, k, it))
//   v    = floor(u * S / 2^64)            (uniform integer in [0, S))
//   next = the first unvisited j, in column order, whose running sum of q
//          exceeds v; when S = 0 (every unvisited p is 0) the lowest
//          unvisited j.
// ---------------------------------------------------------------------------
static int fp32_exponent(float p) {  // floor(log2 p) for p > 0 finite
  uint32_t b;
  std::memcpy(&b, &p, 4);
  int eb = (int)((b >> 23) & 0xFF);
  if (eb) return eb - 127;
  // subnormal: position of the highest set fraction bit
  int e = -127;
  uint32_t f = b & 0x7FFFFFu;
  while (f) {
    ++e;
    f >>= 1;
  }
  return e - 22 - 1;
}

uint64_t orc_rw_quantum(float p, int e) {
  if (!(p > 0.0f)) return 0;
  // p * 2^(40 - e) exactly in fp64 (p has 24 significant bits), then floor
  double v = std::ldexp((double)p, 40 - e);
  return (uint64_t)std::floor(v);
}

int32_t orc_select_rw(const float* row, const uint8_t* visited, int n, uint64_t seed,
                      uint32_t it, uint32_t k, uint32_t t) {
  float pmax = 0.0f;
  int32_t first = -1;
  for (int j = 0; j < n; ++j) {
    if (visited[j]) continue;
    if (first < 0) first = j;
    if (row[j] > pmax) pmax = row[j];
  }
  if (first < 0) return -1;
  if (!(pmax > 0.0f)) return first;
  const int e = fp32_exponent(pmax);
  uint64_t S = 0;
  for (int j = 0; j < n; ++j)
    if (!visited[j]) S += orc_rw_quantum(row[j], e);
  uint32_t ctr[4] = {1u << 30, t, k, it};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  const uint64_t u = ((uint64_t)out[0] << 32) | (uint64_t)out[1];
  const uint64_t v = (uint64_t)(((unsigned __int128)u * (unsigned __int128)S) >> 64);
  uint64_t run = 0;
  for (int j = 0; j < n; ++j) {
    if (visited[j]) continue;
    run += orc_rw_quantum(row[j], e);
    if (run > v) return j;
  }
  return -1;  // unreachable: the running sum reaches S > v
}

static void construct_one_rw(const float* P_val, int n, uint64_t seed, uint32_t it, int k,
                             int32_t* tour) {
  std::vector<uint8_t> visited((size_t)n, 0);
  int32_t cur = orc_start_city(seed, it, (uint32_t)k, n);
  tour[0] = cur;
  visited[cur] = 1;
  for (int t = 1; t < n; ++t) {
    int32_t v = orc_select_rw(P_val + (size_t)cur * n, visited.data(), n, seed, it,
                              (uint32_t)k, (uint32_t)t);
    tour[t] = v;
    visited[v] = 1;
    cur = v;
  }
}

void orc_construct_rw(const float* P_val, int n, uint64_t seed, uint32_t it, int k_begin,
                      int k_end, int32_t* tours, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int k = k_begin; k < k_end; ++k)
    construct_one_rw(P_val, n, seed, it, k, tours + (size_t)(k - k_begin) * n);
  (void)nthreads;
}

// Selection frequencies of independent roulette on one row (the Bernoulli
// trials of the AdaIR visualisation, Sec. 3.3.1): trial tr draws r_j from
// Philox counter (j >> 2, tr mod 2^32, tr div 2^32, salt), word j & 3, and
// the unvisited j maximising fl32(r_j * q_j) (lowest j on ties) wins;
// counts[j] += its wins.
void orc_selection_counts(const float* q, const uint8_t* visited, int n, uint64_t trials,
                          uint64_t seed, uint32_t salt, uint64_t* counts) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint64_t tr = 0; tr < trials; ++tr) {
    int32_t best_j = -1;
    float best = 0.0f;
    for (int j = 0; j < n; ++j) {
      if (visited && visited[j]) continue;
      const uint32_t ctr[4] = {(uint32_t)(j >> 2), (uint32_t)tr, (uint32_t)(tr >> 32), salt};
      uint32_t out[4];
      orc_philox4x32_10(ctr, key, out);
      const float score = orc_uniform(out[j & 3]) * q[j];
      if (best_j < 0 || score > best || (score == best && j < best_j)) {
        best = score;
        best_j = j;
      }
    }
    if (best_j >= 0) counts[best_j] += 1;
  }
}

// Exact summation after Shewchuk, "Adaptive Precision Floating-Point
// Arithmetic" (1997): the running sum is kept as an expansion -- a list of
// non-overlapping doubles of increasing magnitude whose real sum is exactly
// the sum of every input so far.  grow() adds one double with two-sum steps.
static void grow(std::vector<double>& partials, double v) {
  size_t used = 0;
  for (size_t r = 0; r < partials.size(); ++r) {
    double y = partials[r];
    if (std::fabs(v) < std::fabs(y)) std::swap(v, y);
    const double hi = v + y;
    const double lo = y - (hi - v);
    if (lo != 0.0) partials[used++] = lo;
    v = hi;
  }
  partials.resize(used);
  partials.push_back(v);
}

// The double nearest to the real value of an expansion (ties to even): add the
// components from the largest down until a rounding error appears, then settle
// an exact half-way case with the sign of the next component.
static double round_expansion(const std::vector<double>& partials) {
  if (partials.empty()) return 0.0;
  size_t r = partials.size();
  double hi = partials[--r];
  double lo = 0.0;
  while (r > 0) {
    const double v = hi;
    const double y = partials[--r];
    hi = v + y;
    const double yr = hi - v;
    lo = y - yr;
    if (lo != 0.0) break;
  }
  if (r > 0 && ((lo < 0.0 && partials[r - 1] < 0.0) || (lo > 0.0 && partials[r - 1] > 0.0))) {
    const double y = lo * 2.0;
    const double v = hi + y;
    const double yr = v - hi;
    if (y == yr) hi = v;
  }
  return hi;
}

static bool all_finite(const double* x, size_t count) {
  for (size_t q = 0; q < count; ++q)
    if (!std::isfinite(x[q])) return false;
  return true;
}

// The exact sum of count doubles rounded once to double.  Inputs that are not
// all finite give the plain IEEE sum (an infinity or NaN).
static double exact_sum(const double* x, size_t count) {
  if (!all_finite(x, count)) {
    double s = 0.0;
    for (size_t q = 0; q < count; ++q) s = s + x[q];
    return s;
  }
  std::vector<double> partials;
  for (size_t q = 0; q < count; ++q) grow(partials, x[q]);
  return round_expansion(partials);
}

// fp32 value of a double with an infinity read as +-2^128 (the point where
// the fp32 range ends), so that half-way tests work at the overflow boundary.
static double f32_as_double(float f) {
  if (std::isinf(f)) return std::copysign(std::ldexp(1.0, 128), (double)f);
  return (double)f;
}

// The exact sum of count doubles rounded once to fp32 (ties to even).  With h
// the nearest double to the exact sum x, every fp32 value and every point
// half-way between two fp32 neighbours is a double, so rounding h to fp32
// gives the fp32 rounding of x -- except when h is itself such a half-way
// point and x != h; then the sign of x - h (an exact expansion again) picks
// the neighbour.  Inputs that are not all finite give fl32 of the IEEE sum.
static float exact_sum_f32(const double* x, size_t count) {
  if (!all_finite(x, count)) return (float)exact_sum(x, count);
  std::vector<double> partials;
  for (size_t q = 0; q < count; ++q) grow(partials, x[q]);
  const double h = round_expansion(partials);
  float f = (float)h;
  const double fd = f32_as_double(f);
  if (fd != h) {
    const float g = (fd < h) ? std::nextafter(f, INFINITY) : std::nextafter(f, -INFINITY);
    const double gd = f32_as_double(g);
    if (h - fd == gd - h) {  // h lies half-way between f and g
      std::vector<double> rest = partials;
      grow(rest, -h);  // exact x - h
      double sign = 0.0;
      for (double v : rest)
        if (v != 0.0) sign = v;  // the largest component decides the sign
      if ((sign > 0.0 && gd > fd) || (sign < 0.0 && gd < fd)) f = g;
    }
  }
  return f;
}

// The exact sum of count doubles (finite, sum >= 0) rounded once to bfloat16
// (8 significant bits, fp32's exponent range with subnormals down to 2^-133,
// overflow past (2 - 2^-8) 2^127 to +inf; ties to even), returned as the fp32
// value.  As for fp32: every bf16 value and half-way point is a double, so
// rounding h = the nearest double to the sum gives the right answer unless h
// is a half-way point itself, which the sign of the remainder then settles.
static float exact_sum_bf16(const double* x, size_t count) {
  std::vector<double> partials;
  for (size_t q = 0; q < count; ++q) grow(partials, x[q]);
  const double h = round_expansion(partials);
  if (!(h > 0.0)) return 0.0f;
  int e2;
  std::frexp(h, &e2);                      // h = f 2^e2, f in [0.5, 1)
  const int sh = std::max(e2 - 1, -126) - 7;  // exponent of the bf16 quantum at h
  const double y = std::ldexp(h, -sh);     // exact
  const double fl = std::floor(y);
  double r;
  if (y - fl == 0.5) {
    std::vector<double> rest = partials;
    grow(rest, -h);
    double sign = 0.0;
    for (double v : rest)
      if (v != 0.0) sign = v;
    if (sign > 0.0)
      r = fl + 1.0;
    else if (sign < 0.0)
      r = fl;
    else
      r = std::fmod(fl, 2.0) == 0.0 ? fl : fl + 1.0;
  } else {
    r = std::nearbyint(y);  // round half to even (the default mode)
  }
  const double v = std::ldexp(r, sh);
  if (v >= 0x1p128) return INFINITY;
  return (float)v;
}

float orc_exact_sum_bf16(const double* x, int64_t count) { return exact_sum_bf16(x, (size_t)count); }

// f(s) (Eq. 3): the closed tour length, the sum over t = 0..n-1 of
// d(p_t, p_{t+1 mod n}).  Eq. 3 writes f as a plain sum and fixes no order,
// so none is imposed: the n fp64 edge lengths are summed exactly and the sum
// is rounded once to fp64 (ties to even).
void orc_tour_lengths(const double* D, int n, const int32_t* tours, int m, double* L) {
  std::vector<double> edges((size_t)n);
  for (int k = 0; k < m; ++k) {
    const int32_t* p = tours + (size_t)k * n;
    for (int t = 0; t < n; ++t) edges[t] = D[(size_t)p[t] * n + p[(t + 1) % n]];
    L[k] = exact_sum(edges.data(), (size_t)n);
  }
}

// Eq. 2: the path and its one-step cyclic shift side by side, row t = (p_t, p_{t-1}).
void orc_index_matrix(const int32_t* tour, int n, int32_t* I) {
  for (int t = 0; t < n; ++t) {
    I[2 * t] = tour[t];
    I[2 * t + 1] = tour[(t + n - 1) % n];
  }
}

// Evaporation then deposit (Sec. 2.3, Eq. 3 with weight Q / f):
//   c_k = fl64(Q / L_k);
//   A^(k)_ij = c_k if (i,j) or (j,i) is a row of I^(k), else 0;
//   tau'_ij = fl32(keep * tau_ij) with keep = fl32(1 - rho)      (fp32 tensor)
//   tau_ij <- tau'_ij + sum over paths of A^(k)_ij, the real sum rounded once
//             to fp32 (ties to even); tau'_ij where no path has the edge.
static void deposit_rounded(float* tau, int n, const int32_t* tours, const double* L, int m,
                            float rho, float Q, bool bf16);

void orc_deposit(float* tau, int n, const int32_t* tours, const double* L, int m,
                 float rho, float Q) {
  deposit_rounded(tau, n, tours, L, m, rho, Q, false);
}

// As orc_deposit with M_tau stored in bfloat16: the same exact sum
// fl32(keep * tau) + sum of c_k is rounded once to bf16; entries no path
// uses become the bf16 rounding of fl32(keep * tau).
void orc_deposit_tau_bf16(float* tau, int n, const int32_t* tours, const double* L, int m,
                          float rho, float Q) {
  deposit_rounded(tau, n, tours, L, m, rho, Q, true);
}

static void deposit_rounded(float* tau, int n, const int32_t* tours, const double* L, int m,
                            float rho, float Q, bool bf16) {
  // every (entry, weight) pair, grouped by entry
  std::vector<std::pair<size_t, double>> items;
  items.reserve((size_t)2 * n * m);
  std::vector<int32_t> I((size_t)2 * n);
  for (int k = 0; k < m; ++k) {
    double c = (double)Q / L[k];
    orc_index_matrix(tours + (size_t)k * n, n, I.data());
    for (int t = 0; t < n; ++t) {
      int32_t a = I[2 * t], b = I[2 * t + 1];
      items.emplace_back((size_t)a * n + b, c);
      items.emplace_back((size_t)b * n + a, c);
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<size_t, double>& x, const std::pair<size_t, double>& y) {
                     return x.first < y.first;
                   });
  const float keep = 1.0f - rho;
  for (size_t e = 0; e < (size_t)n * n; ++e) tau[e] = keep * tau[e];
  std::vector<uint8_t> touched(bf16 ? (size_t)n * n : 0, 0);
  std::vector<double> group;
  for (size_t q = 0; q < items.size();) {
    const size_t e = items[q].first;
    group.assign(1, (double)tau[e]);
    while (q < items.size() && items[q].first == e) group.push_back(items[q++].second);
    tau[e] = bf16 ? exact_sum_bf16(group.data(), group.size()) : exact_sum_f32(group.data(), group.size());
    if (bf16) touched[e] = 1;
  }
  if (bf16)
    for (size_t e = 0; e < (size_t)n * n; ++e)
      if (!touched[e]) tau[e] = orc_from_bf16(orc_to_bf16(tau[e]));
}

// Sec. 2.3 (tensorization of ant paths): the solution set is sorted by
// fitness -- tour length ascending, equal lengths by ant index -- and the
// first k paths are selected.  selected[k] = 1 for them.  k <= 0 or k >= m
// selects every path (plain Ant System).
void orc_select_topk(const double* L, int m, int k, uint8_t* selected) {
  std::vector<int> order((size_t)m);
  for (int q = 0; q < m; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return L[a] < L[b]; });
  const int take = (k <= 0 || k >= m) ? m : k;
  for (int q = 0; q < m; ++q) selected[q] = 0;
  for (int q = 0; q < take; ++q) selected[order[q]] = 1;
}

// Evaporation then the deposit of the k selected paths only (Sec. 2.3:
// Delta M_tau sums A over the selected set P); every entry evaporates.
static void deposit_topk_impl(float* tau, int n, const int32_t* tours, const double* L, int m,
                              float rho, float Q, int k, bool bf16);

void orc_deposit_topk(float* tau, int n, const int32_t* tours, const double* L, int m,
                      float rho, float Q, int k) {
  deposit_topk_impl(tau, n, tours, L, m, rho, Q, k, false);
}

static void deposit_topk_impl(float* tau, int n, const int32_t* tours, const double* L, int m,
                              float rho, float Q, int k, bool bf16) {
  std::vector<uint8_t> sel((size_t)m);
  orc_select_topk(L, m, k, sel.data());
  std::vector<int32_t> st;
  std::vector<double> sl;
  for (int q = 0; q < m; ++q) {
    if (!sel[q]) continue;
    st.insert(st.end(), tours + (size_t)q * n, tours + (size_t)(q + 1) * n);
    sl.push_back(L[q]);
  }
  deposit_rounded(tau, n, st.data(), sl.data(), (int)sl.size(), rho, Q, bf16);
}

double orc_exact_sum(const double* x, int64_t count) { return exact_sum(x, (size_t)count); }
float orc_exact_sum_f32(const double* x, int64_t count) { return exact_sum_f32(x, (size_t)count); }

void orc_deposit_fp32_order(float* tau, int n, const int32_t* tours, const double* L,
                            int m, float rho, float Q, const int64_t* perm) {
  const float keep = 1.0f - rho;
  for (size_t e = 0; e < (size_t)n * n; ++e) tau[e] = keep * tau[e];
  int64_t total = (int64_t)2 * m * n;
  for (int64_t q = 0; q < total; ++q) {
    int64_t id = perm ? perm[q] : q;
    int64_t k = id / (2 * (int64_t)n);
    int64_t rest = id % (2 * (int64_t)n);
    int64_t t = rest / 2;
    int dir = (int)(rest % 2);
    const int32_t* p = tours + (size_t)k * n;
    int32_t a = p[t], b = p[(t + n - 1) % n];
    if (dir) {
      int32_t tmp = a;
      a = b;
      b = tmp;
    }
    float c = (float)((double)Q / L[k]);
    tau[(size_t)a * n + b] = tau[(size_t)a * n + b] + c;
  }
}

void orc_init_tau(float* tau, int n, float tau0) {
  for (size_t e = 0; e < (size_t)n * n; ++e) tau[e] = tau0;
}

// Iterations it0 .. it0+iters-1 of the whole path.  The iteration best is the
// shortest tour (lowest ant index on ties); the global best is replaced only
// by a strictly shorter tour.
void orc_run(const orc_params* prm, const double* D, const float* H, float* tau,
             uint32_t it0, int iters, int32_t* best_tour, double* best_len,
             int32_t* last_tours, double* last_L, int nthreads) {
  const int n = prm->n, m = prm->m;
  std::vector<float> P((size_t)n * n);
  std::vector<int32_t> tours((size_t)m * n);
  std::vector<double> L((size_t)m);
  for (int q = 0; q < iters; ++q) {
    uint32_t it = it0 + (uint32_t)q;
    float inv_gamma = 1.0f;
    if (prm->adair) {
      float g = orc_gamma((int)it, prm->gamma_T, prm->gamma_max, prm->gamma_min);
      inv_gamma = orc_inv_gamma(g);
    }
    orc_build_P(tau, H, n, prm->alpha, inv_gamma, prm->prec, P.data(), nullptr, nullptr);
    if (prm->rw)
      orc_construct_rw(P.data(), n, prm->seed, it, 0, m, tours.data(), nthreads);
    else
      orc_construct(P.data(), n, prm->seed, it, 0, m, tours.data(), nthreads);
    orc_tour_lengths(D, n, tours.data(), m, L.data());
    int kb = 0;
    for (int k = 1; k < m; ++k)
      if (L[k] < L[kb]) kb = k;
    if (L[kb] < *best_len) {
      *best_len = L[kb];
      std::memcpy(best_tour, tours.data() + (size_t)kb * n, sizeof(int32_t) * n);
    }
    deposit_topk_impl(tau, n, tours.data(), L.data(), m, prm->rho, prm->Q, prm->topk, prm->tau_bf16 != 0);
  }
  if (last_tours) std::memcpy(last_tours, tours.data(), sizeof(int32_t) * tours.size());
  if (last_L) std::memcpy(last_L, L.data(), sizeof(double) * L.size());
}

}  // extern "C"
