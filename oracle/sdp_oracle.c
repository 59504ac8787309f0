/*
 * sdp_oracle.c -- plain, slow, FP64 CPU oracle for the scenario-batched
 * Bellman updates of arXiv 2602.05179 (Split for CVRPSD and the
 * order-up-to inventory-reinsertion DP).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library; both sides receive the same input arrays.
 *
 * Every function follows the paper's definitions literally, in double
 * precision, without blocking, prefix-sum tricks or any reordering beyond what
 * the definitions state:
 *
 *   - oracle_minplus_matvec: the min-plus matrix-vector Bellman update
 *       J_{t+1}(j) = min_i { A(i,j) + J_t(i) }   (Sec. 2, "Min-Plus Matrix
 *       Formulation"; worked example in Appendix "Illustrative example for the
 *       min-plus matrix-vector Bellman update").
 *   - oracle_split: Split DP of Sec. 2 "Instantiation A" (Eq. eqdpA):
 *       J(0)=0, J(i) = min_{p<i} J(p) + A(p,i), A(p,i) = W(p,i) if the route
 *       sigma_{p+1..i} has load <= Q, +inf otherwise, with
 *       W(p,i) = c(0,s_{p+1}) + sum_{k=p+1}^{i-1} c(s_k,s_{k+1}) + c(s_i,n+1).
 *   - oracle_split_soft: the same DP with the penalised (soft) capacity of
 *       the paper's CVRPSD model: every split allowed, beta per unit of route
 *       load above Q added to W.
 *   - oracle_split_matrix: the same DP through the explicit masked matrix A
 *       (Appendix "Illustrative Matrix Form of DP" for Split), one scenario.
 *   - oracle_split_route_counts: backtrack of the optimal split and the
 *       arc-usage counts; the route cost is linear in the travel costs, so the
 *       gradient of the scenario mean w.r.t. c(a,b) is the mean usage count.
 *   - oracle_reinsert: backward DP of Algorithm "SolveBatchDP" (C[T]=0, then
 *       for t=T-1..0 compare no delivery with delivery up to U, record the
 *       decision) and the backtrack from the initial inventory.
 *   - oracle_reinsert_routes: the same backward DP with several candidate
 *       route options per day (an entry of A is a minimum over routes).
 *   - oracle_reinsert_forward: forward min-plus recursion of Eq. eqdp2 with
 *       the transition matrix A^{t}(I,J) of Sec. 2 "Instantiation B" built
 *       explicitly and multiplied with oracle_minplus_matvec.
 *
 * Readings of points the paper leaves open (S1..S10, R1..R9 in the design
 * notes) are stated next to the code that takes them.
 *
 * Pins: the worked examples of the paper (min-plus toy, Split toy, inventory
 * toy), brute-force enumeration of all splits (n<=10) and all delivery
 * sequences (T<=8), closed forms and invariants -- see tests/.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_VERSION 1

int oracle_version(void) { return ORACLE_VERSION; }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Generic min-plus matrix-vector product (Sec. 2, Min-Plus Matrix
 * Formulation).  A is m x k row-major, A[i*k + j] = A(i,j) (row = state at t,
 * column = state at t+1), +inf marks an infeasible transition.  out[j] =
 * min_i A(i,j) + J[i]; argmin_out[j] (optional) = smallest i attaining it, or
 * -1 when every entry of the column is +inf. */
void oracle_minplus_matvec(int m, int k, const double* A, const double* J,
                           double* out, int32_t* argmin_out) {
  for (int j = 0; j < k; ++j) {
    double best = INFINITY;
    int32_t arg = -1;
    for (int i = 0; i < m; ++i) {
      double a = A[(size_t)i * k + j];
      if (isinf(a) || isinf(J[i])) continue; /* +inf masking: no inf+x */
      double v = a + J[i];
      if (v < best) { best = v; arg = i; }
    }
    out[j] = best;
    if (argmin_out) argmin_out[j] = arg;
  }
}

/* ------------------------------------------------------------------------ */
/* Travel cost c(a,b) for nodes a,b in 0..n (0 = depot).  Reading S1: the
 * destination depot n+1 is the same location as the departure depot 0.
 * Reading S8: with coordinates, c is the Euclidean distance in FP64 of the
 * FP32 coordinates; with a matrix, c(a,b) = dist[a*(n+1)+b] read as FP64. */
typedef struct {
  int n;
  const float* coords; /* [(n+1)*2] or NULL */
  const float* dist;   /* [(n+1)*(n+1)] or NULL */
} cost_t;

static double cost_ab(const cost_t* c, int a, int b) {
  if (c->dist) return (double)c->dist[(size_t)a * (c->n + 1) + b];
  double dx = (double)c->coords[2 * a] - (double)c->coords[2 * b];
  double dy = (double)c->coords[2 * a + 1] - (double)c->coords[2 * b + 1];
  return sqrt(dx * dx + dy * dy);
}

/* Split, one scenario.  q_by_customer[c-1] = demand of customer c (reading
 * S2: demands are indexed by customer id; the tour permutes them).
 * J is scratch of n+1 doubles.  Returns J(n) (+inf if some customer's demand
 * exceeds Q, reading S3).  pred[i-1] = argmin p of J(i) (smallest p on exact
 * ties, reading S4), -1 when J(i) is +inf.  margin[i-1] = (second-best
 * candidate - best) / |best| over feasible predecessors, +inf when only one
 * candidate exists.  *arcs = number of capacity-feasible pairs (p,i), p<i. */
static double split_one(int n, const int32_t* tour, const cost_t* c, int32_t Q,
                        const int32_t* q_by_customer, double* J,
                        int32_t* pred, double* margin, int64_t* arcs) {
  int64_t narcs = 0;
  J[0] = 0.0;
  for (int i = 1; i <= n; ++i) {
    double best = INFINITY, second = INFINITY;
    int32_t bestp = -1;
    int64_t load = 0;
    double inner = 0.0; /* sum_{k=p+1}^{i-1} c(s_k, s_{k+1}) */
    const int si = tour[i - 1];
    const double back = cost_ab(c, si, 0); /* c(s_i, n+1) */
    for (int p = i - 1; p >= 0; --p) {
      const int sp1 = tour[p]; /* s_{p+1} */
      load += q_by_customer[sp1 - 1];
      if (load > Q) break; /* A(p,i) = +inf for this p and every smaller p */
      ++narcs;
      if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);
      if (isinf(J[p])) continue;
      const double W = cost_ab(c, 0, sp1) + inner + back;
      const double cand = J[p] + W;
      /* p runs downwards, so "<=" keeps the smallest p on exact ties. */
      if (cand <= best) {
        if (bestp >= 0) second = best < second ? best : second;
        best = cand;
        bestp = p;
      } else if (cand < second) {
        second = cand;
      }
    }
    J[i] = best;
    if (pred) pred[i - 1] = bestp;
    if (margin) {
      if (bestp < 0 || isinf(second)) margin[i - 1] = INFINITY;
      else margin[i - 1] = (second - best) / fmax(fabs(best), 1e-300);
    }
  }
  if (arcs) *arcs = narcs;
  return J[n];
}

/* Split over S scenarios.  Exactly one of coords/dist is non-NULL.
 * demands[s*n + (c-1)] = demand of customer c in scenario s.
 * cost_out[s] = J_s(n) in FP64; pred_out/margin_out [S*n] and arcs_out [S]
 * are optional.  mean_out (optional) = (1/S) sum_s cost_out[s], summed
 * sequentially in scenario order (the expectation of Sec. 2 / the SAA mean).
 * Returns 0, or -1 on a bad argument. */
int oracle_split(int n, const int32_t* tour, const float* coords,
                 const float* dist, int32_t Q, int64_t S,
                 const int32_t* demands, double* cost_out, int32_t* pred_out,
                 double* margin_out, int64_t* arcs_out, double* mean_out,
                 int nthreads) {
  if (n < 0 || S < 0 || Q <= 0 || !cost_out) return -1;
  if ((coords == NULL) == (dist == NULL) && n > 0) return -1;
  cost_t c = {n, coords, dist};
  int bad = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
#endif
  {
    double* J = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    if (!J) bad = 1;
    else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t s = 0; s < S; ++s) {
        int64_t a = 0;
        cost_out[s] = split_one(n, tour, &c, Q, demands + s * n, J,
                                pred_out ? pred_out + s * n : NULL,
                                margin_out ? margin_out + s * n : NULL, &a);
        if (arcs_out) arcs_out[s] = a;
      }
      free(J);
    }
  }
  if (bad) return -2;
  if (mean_out) {
    double sum = 0.0;
    for (int64_t s = 0; s < S; ++s) sum += cost_out[s];
    *mean_out = S > 0 ? sum / (double)S : 0.0;
  }
  return 0;
}

/* Fleet-limited Split, one scenario (Appendix A, extensive model: constraint
 * eq:fleet_size allows at most K vehicles, i.e. at most K routes; the
 * giant-tour example with "three vehicles available").  Reading F1: hard
 * capacity as in Eq. eqdpA, at most K routes.  With J_k(i) the cost of
 * serving positions 1..i with exactly k routes:
 *     J_0(0) = 0,  J_0(i) = +inf (i > 0),  J_k(0) = +inf (k > 0),
 *     J_k(i) = min over capacity-feasible p < i of J_{k-1}(p) + W(p,i),
 * and cost = min_{1 <= k <= K} J_k(n) (n = 0: cost 0, no route).  Ties: the
 * smallest p at every (k, i) (reading S4), then the fewest routes.  J and M
 * are scratch [(K+1)*(n+1)] doubles, P [(K+1)*(n+1)] int32 (the argmin p).
 * *nroutes = routes of the optimal split (0 when infeasible); route[i-1] =
 * index of the route serving position i (0-based, in tour order), -1 when
 * infeasible.  *margin = min over the choices along the optimal split (each
 * argmin p, and the choice of k) of (second best - best) / |best|, +inf when
 * every choice had a single candidate. */
static double split_fleet_one(int n, const int32_t* tour, const cost_t* c, int32_t Q, int K,
                              const int32_t* q_by_customer, double* J, int32_t* P,
                              double* M, int32_t* nroutes, int32_t* route, double* margin) {
  const int w = n + 1;
  for (int k = 0; k <= K; ++k)
    for (int i = 0; i <= n; ++i) {
      J[k * w + i] = INFINITY;
      P[k * w + i] = -1;
      M[k * w + i] = INFINITY;
    }
  J[0] = 0.0;
  for (int k = 1; k <= K; ++k) {
    for (int i = 1; i <= n; ++i) {
      double best = INFINITY, second = INFINITY;
      int32_t bestp = -1;
      int64_t load = 0;
      double inner = 0.0; /* sum_{m=p+1}^{i-1} c(s_m, s_{m+1}) */
      const double back = cost_ab(c, tour[i - 1], 0);
      for (int p = i - 1; p >= 0; --p) {
        const int sp1 = tour[p];
        load += q_by_customer[sp1 - 1];
        if (load > Q) break;
        if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);
        const double prev = J[(k - 1) * w + p];
        if (isinf(prev)) continue;
        const double cand = prev + (cost_ab(c, 0, sp1) + inner + back);
        if (cand <= best) {  /* p runs downwards: "<=" keeps the smallest p */
          if (bestp >= 0) second = best < second ? best : second;
          best = cand;
          bestp = p;
        } else if (cand < second) {
          second = cand;
        }
      }
      J[k * w + i] = best;
      P[k * w + i] = bestp;
      M[k * w + i] = (bestp < 0 || isinf(second)) ? INFINITY
                                                  : (second - best) / fmax(fabs(best), 1e-300);
    }
  }
  if (n == 0) {
    *nroutes = 0;
    *margin = INFINITY;
    return 0.0;
  }
  double best = INFINITY, second = INFINITY;
  int bestk = 0;
  for (int k = 1; k <= K; ++k) {
    const double v = J[k * w + n];
    if (v < best) {  /* "<": the fewest routes on ties */
      second = best;
      best = v;
      bestk = k;
    } else if (v < second) {
      second = v;
    }
  }
  double mg = (bestk == 0 || isinf(second)) ? INFINITY : (second - best) / fmax(fabs(best), 1e-300);
  *nroutes = bestk;
  if (bestk == 0) {
    if (route)
      for (int i = 0; i < n; ++i) route[i] = -1;
    *margin = INFINITY;
    return INFINITY;
  }
  int i = n, k = bestk;
  while (i > 0) {
    const int p = P[k * w + i];
    mg = fmin(mg, M[k * w + i]);
    if (route)
      for (int m = p; m < i; ++m) route[m] = k - 1;
    i = p;
    --k;
  }
  *margin = mg;
  return best;
}

/* Fleet-limited Split over S scenarios (arguments as oracle_split, plus K >=
 * 1).  cost_out [S] FP64 (+inf where no split into at most K routes fits the
 * capacity); nroutes_out [S], route_out [S*n], margin_out [S] optional;
 * mean_out as in oracle_split.  Returns 0, -1 on a bad argument, -2 when out
 * of memory. */
int oracle_split_fleet(int n, const int32_t* tour, const float* coords, const float* dist,
                       int32_t Q, int K, int64_t S, const int32_t* demands, double* cost_out,
                       int32_t* nroutes_out, int32_t* route_out, double* margin_out,
                       double* mean_out, int nthreads) {
  if (n < 0 || S < 0 || Q <= 0 || K < 1 || !cost_out) return -1;
  if ((coords == NULL) == (dist == NULL) && n > 0) return -1;
  cost_t c = {n, coords, dist};
  int bad = 0;
  const size_t cells = (size_t)(K + 1) * (size_t)(n + 1);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
#endif
  {
    double* J = (double*)malloc(sizeof(double) * cells);
    double* M = (double*)malloc(sizeof(double) * cells);
    int32_t* P = (int32_t*)malloc(sizeof(int32_t) * cells);
    if (!J || !M || !P) bad = 1;
    else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t s = 0; s < S; ++s) {
        int32_t nr = 0;
        double mg = INFINITY;
        cost_out[s] = split_fleet_one(n, tour, &c, Q, K, demands + s * n, J, P, M, &nr,
                                      route_out ? route_out + s * n : NULL, &mg);
        if (nroutes_out) nroutes_out[s] = nr;
        if (margin_out) margin_out[s] = mg;
      }
    }
    free(J);
    free(M);
    free(P);
  }
  if (bad) return -2;
  if (mean_out) {
    double sum = 0.0;
    for (int64_t s = 0; s < S; ++s) sum += cost_out[s];
    *mean_out = S > 0 ? sum / (double)S : 0.0;
  }
  return 0;
}

/* Soft-capacity Split, one scenario (the penalised route load of the
 * paper's CVRPSD model, Sec. "MILP formulation": a route whose load exceeds
 * the capacity pays beta per unit of excess, l_k >= load_k - C, l_k >= 0, in
 * the objective).  Every split is allowed:
 *   J(0) = 0,  J(i) = min_{0<=p<i} J(p) + W(p,i) + beta * max(0, load(s_{p+1..i}) - Q),
 * W as in split_one.  Service times add the same constant to every split and
 * are left out; the fleet is unlimited (reading S6).  Ties: smallest p.
 * margin as in split_one; *arcs = i(i+1)/2 summed, every pair (p,i). */
static double split_soft_one(int n, const int32_t* tour, const cost_t* c, int32_t Q,
                             double beta, const int32_t* q_by_customer, double* J,
                             int32_t* pred, double* margin, int64_t* arcs) {
  int64_t narcs = 0;
  J[0] = 0.0;
  for (int i = 1; i <= n; ++i) {
    double best = INFINITY, second = INFINITY;
    int32_t bestp = -1;
    int64_t load = 0;
    double inner = 0.0; /* sum_{k=p+1}^{i-1} c(s_k, s_{k+1}) */
    const int si = tour[i - 1];
    const double back = cost_ab(c, si, 0);
    for (int p = i - 1; p >= 0; --p) {
      const int sp1 = tour[p];
      load += q_by_customer[sp1 - 1];
      ++narcs;
      if (p < i - 1) inner += cost_ab(c, sp1, tour[p + 1]);
      const double W = cost_ab(c, 0, sp1) + inner + back;
      const double excess = load > Q ? (double)(load - Q) : 0.0;
      const double cand = J[p] + W + beta * excess;
      if (cand <= best) { /* p runs downwards: "<=" keeps the smallest p */
        if (bestp >= 0) second = best < second ? best : second;
        best = cand;
        bestp = p;
      } else if (cand < second) {
        second = cand;
      }
    }
    J[i] = best;
    if (pred) pred[i - 1] = bestp;
    if (margin) {
      if (bestp < 0 || isinf(second)) margin[i - 1] = INFINITY;
      else margin[i - 1] = (second - best) / fmax(fabs(best), 1e-300);
    }
  }
  if (arcs) *arcs = narcs;
  return J[n];
}

/* Soft-capacity Split over S scenarios (arguments as oracle_split, plus the
 * penalty beta per unit of load above Q). */
int oracle_split_soft(int n, const int32_t* tour, const float* coords, const float* dist,
                      int32_t Q, double beta, int64_t S, const int32_t* demands,
                      double* cost_out, int32_t* pred_out, double* margin_out,
                      int64_t* arcs_out, double* mean_out, int nthreads) {
  if (n < 0 || S < 0 || Q <= 0 || !cost_out || !(beta >= 0.0)) return -1;
  if ((coords == NULL) == (dist == NULL) && n > 0) return -1;
  cost_t c = {n, coords, dist};
  int bad = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
#endif
  {
    double* J = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    if (!J) bad = 1;
    else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
      for (int64_t s = 0; s < S; ++s) {
        int64_t a = 0;
        cost_out[s] = split_soft_one(n, tour, &c, Q, beta, demands + s * n, J,
                                     pred_out ? pred_out + s * n : NULL,
                                     margin_out ? margin_out + s * n : NULL, &a);
        if (arcs_out) arcs_out[s] = a;
      }
      free(J);
    }
  }
  if (bad) return -2;
  if (mean_out) {
    double sum = 0.0;
    for (int64_t s = 0; s < S; ++s) sum += cost_out[s];
    *mean_out = S > 0 ? sum / (double)S : 0.0;
  }
  return 0;
}

/* Split of one scenario through the explicit masked matrix A (Appendix
 * "Illustrative Matrix Form of DP"): A_out[(p)*(n+1) + i] = W(p,i) when p<i
 * and the load of s_{p+1..i} is <= Q, +inf otherwise (including p>=i).
 * Then J(0)=0 and, column by column, J(i) = min-plus of column i of A with
 * J(0..i-1).  V_out = (J(0),...,J(n)). */
int oracle_split_matrix(int n, const int32_t* tour, const float* coords,
                        const float* dist, int32_t Q,
                        const int32_t* q_by_customer, double* A_out,
                        double* V_out) {
  if (n < 0 || Q <= 0) return -1;
  cost_t c = {n, coords, dist};
  const int m = n + 1;
  for (int p = 0; p < m; ++p)
    for (int i = 0; i < m; ++i) {
      double a = INFINITY;
      if (p < i) {
        int64_t load = 0;
        for (int k = p + 1; k <= i; ++k) load += q_by_customer[tour[k - 1] - 1];
        if (load <= Q) {
          double w = cost_ab(&c, 0, tour[p]);
          for (int k = p + 1; k <= i - 1; ++k)
            w += cost_ab(&c, tour[k - 1], tour[k]);
          w += cost_ab(&c, tour[i - 1], 0);
          a = w;
        }
      }
      A_out[(size_t)p * m + i] = a;
    }
  V_out[0] = 0.0;
  double* col = (double*)malloc(sizeof(double) * (size_t)m);
  if (!col) return -2;
  for (int i = 1; i < m; ++i) {
    for (int p = 0; p < i; ++p) col[p] = A_out[(size_t)p * m + i];
    double r;
    oracle_minplus_matvec(i, 1, col, V_out, &r, NULL);
    V_out[i] = r;
  }
  free(col);
  return 0;
}

/* Backtrack of the optimal splits and arc-usage counts.  From pred[s*n+i-1]
 * (as produced by oracle_split), walk i = n -> pred -> ... -> 0; each route
 * p+1..i starts at tour position p+1 and ends at position i.
 *   start_cnt[k-1] = #scenarios in which a route starts at position k,
 *   end_cnt[k-1]   = #scenarios in which a route ends at position k.
 * Scenarios whose chain is broken (pred -1: infeasible) are skipped and
 * counted in *skipped.  Returns 0. */
int oracle_split_route_counts(int n, int64_t S, const int32_t* pred,
                              int64_t* start_cnt, int64_t* end_cnt,
                              int64_t* skipped) {
  memset(start_cnt, 0, sizeof(int64_t) * (size_t)n);
  memset(end_cnt, 0, sizeof(int64_t) * (size_t)n);
  int64_t skip = 0;
  for (int64_t s = 0; s < S; ++s) {
    const int32_t* ps = pred + s * n;
    int ok = 1;
    for (int i = n; i > 0;) {
      int p = ps[i - 1];
      if (p < 0 || p >= i) { ok = 0; break; }
      i = p;
    }
    if (!ok) { ++skip; continue; }
    for (int i = n; i > 0;) {
      int p = ps[i - 1];
      start_cnt[p] += 1; /* route starts at position p+1 */
      end_cnt[i - 1] += 1;
      i = p;
    }
  }
  if (skipped) *skipped = skip;
  return 0;
}

/* Gradient of the scenario mean of the optimal split cost with respect to the
 * travel-cost matrix, at a point where each scenario's optimum is unique: each
 * route p+1..i uses arcs (0,s_{p+1}), (s_k,s_{k+1}) for p+1<=k<i and
 * (s_i,0), each once, so d mean / d c(a,b) = (1/S) * #uses of (a,b).
 * grad_out[(n+1)*(n+1)] row-major is overwritten. */
int oracle_split_mean_grad(int n, const int32_t* tour, int64_t S,
                           const int32_t* pred, double* grad_out) {
  const int m = n + 1;
  memset(grad_out, 0, sizeof(double) * (size_t)m * m);
  int64_t used = 0;
  for (int64_t s = 0; s < S; ++s) {
    const int32_t* ps = pred + s * n;
    int ok = 1;
    for (int i = n; i > 0;) {
      int p = ps[i - 1];
      if (p < 0 || p >= i) { ok = 0; break; }
      i = p;
    }
    if (!ok) continue;
    ++used;
    for (int i = n; i > 0;) {
      int p = ps[i - 1];
      grad_out[(size_t)0 * m + tour[p]] += 1.0;
      for (int k = p + 1; k < i; ++k)
        grad_out[(size_t)tour[k - 1] * m + tour[k]] += 1.0;
      grad_out[(size_t)tour[i - 1] * m + 0] += 1.0;
      i = p;
    }
  }
  (void)used;
  if (S > 0)
    for (size_t e = 0; e < (size_t)m * m; ++e) grad_out[e] /= (double)S;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Inventory reinsertion under an order-up-to policy (Sec. 2 Instantiation B,
 * Appendix "Evaluation on Instantiation B", Algorithm SolveBatchDP).
 *
 * One customer; inventory states I = 0..U (start-of-day inventory, reading
 * R8); days t = 0..T-1 (0-based) with consumption d_t = cons[s*T + t] and
 * routing data fixed[t].  Actions q in {0, U-I} (OU policy); delivery arrives
 * before consumption and unmet demand is lost (reading R3):
 *     end inventory J = max(0, I + q - d_t).
 * Stage cost (reading R1):  F_t(q) + e(I + q - d_t), where
 *     F_t(q) = fixed[t] + unit_cost * q  if q > 0, and 0 if q = 0 (reading R2),
 *     e(x)   = h * x for x >= 0 (holding) and p * (-x) for x < 0 (lost-sales
 *              penalty per unit), or, in table mode, e(x) = H[max(0,x)] (the
 *              end-of-day cost as a function of end inventory only, as in the
 *              paper's inventory toy).
 * Terminal cost C_T = 0 (reading R5).  Ties prefer no delivery (reading R6). */
typedef struct {
  int T, U;
  double h, p, unit_cost;
  const float* fixed;  /* [T] */
  const double* H;     /* [U+1] or NULL */
} inv_t;

static double end_cost(const inv_t* m, int64_t x) {
  if (m->H) return m->H[x > 0 ? (x > m->U ? m->U : x) : 0];
  return x >= 0 ? m->h * (double)x : m->p * (double)(-x);
}

static double route_cost(const inv_t* m, int t, int q) {
  return q > 0 ? (double)m->fixed[t] + m->unit_cost * (double)q : 0.0;
}

/* Backward DP for one scenario.  C is scratch [(T+1)*(U+1)], dec is scratch
 * [T*(U+1)], marg (optional) [T*(U+1)] = |dv-nd|/max(|nd|,|dv|) (+inf when
 * only one action exists, i.e. I = U).  Returns C_0(I0). */
static double reinsert_one(const inv_t* m, int I0, const int32_t* d,
                           double* C, uint8_t* dec, double* marg,
                           uint8_t* policy, double* value0) {
  const int T = m->T, U = m->U, W = U + 1;
  for (int I = 0; I < W; ++I) C[(size_t)T * W + I] = 0.0;
  for (int t = T - 1; t >= 0; --t) {
    const int64_t dt = d[t];
    const double* Cn = C + (size_t)(t + 1) * W;
    double* Ct = C + (size_t)t * W;
    for (int I = 0; I < W; ++I) {
      /* no delivery: q = 0 */
      int64_t x0 = (int64_t)I - dt;
      double nd = end_cost(m, x0) + Cn[x0 > 0 ? x0 : 0];
      double best = nd;
      uint8_t a = 0;
      double mg = INFINITY;
      if (I < U) { /* deliver up to U: q = U - I */
        int q = U - I;
        int64_t x1 = (int64_t)I + q - dt;
        double dv = route_cost(m, t, q) + end_cost(m, x1) + Cn[x1 > 0 ? x1 : 0];
        if (dv < nd) { best = dv; a = 1; }
        double den = fmax(fabs(nd), fabs(dv));
        mg = den > 0 ? fabs(dv - nd) / den : (dv == nd ? 0.0 : INFINITY);
      }
      Ct[I] = best;
      dec[(size_t)t * W + I] = a;
      if (marg) marg[(size_t)t * W + I] = mg;
    }
  }
  if (value0)
    for (int I = 0; I < W; ++I) value0[I] = C[I];
  if (policy) {
    int64_t I = I0;
    for (int t = 0; t < T; ++t) {
      uint8_t a = dec[(size_t)t * W + I];
      policy[t] = a;
      int64_t q = a ? (U - I) : 0;
      int64_t x = I + q - d[t];
      I = x > 0 ? x : 0;
    }
  }
  return C[I0];
}

/* Backward DP + backtrack over S scenarios.  fixed[T] = per-day routing cost
 * f_t (shared by all scenarios); H (optional, [U+1]) switches to table mode.
 * value_out[s] = C_0(I0); policy_out[s*T+t] (optional) = decision on day t
 * along the optimal path from I0; value0_out[s*(U+1)+I] (optional) = C_0(I);
 * margin_out[s*T*(U+1) + t*(U+1) + I] (optional) = relative gap between the
 * two actions at (t, I).  mean_out (optional) = sequential FP64 mean. */
int oracle_reinsert(int T, int U, int I0, double h, double p, double unit_cost,
                    const float* fixed, const double* H, int64_t S,
                    const int32_t* cons, double* value_out,
                    uint8_t* policy_out, double* value0_out,
                    double* margin_out, double* mean_out, int nthreads) {
  if (T <= 0 || U < 0 || I0 < 0 || I0 > U || S < 0 || !value_out || !fixed)
    return -1;
  inv_t m = {T, U, h, p, unit_cost, fixed, H};
  const size_t W = (size_t)U + 1;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
#endif
  {
    double* C = (double*)malloc(sizeof(double) * (size_t)(T + 1) * W);
    uint8_t* dec = (uint8_t*)malloc((size_t)T * W);
    if (!C || !dec) bad = 1;
    else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t s = 0; s < S; ++s) {
        value_out[s] = reinsert_one(
            &m, I0, cons + s * T, C, dec,
            margin_out ? margin_out + (size_t)s * T * W : NULL,
            policy_out ? policy_out + s * T : NULL,
            value0_out ? value0_out + (size_t)s * W : NULL);
      }
    }
    free(C);
    free(dec);
  }
  if (bad) return -2;
  if (mean_out) {
    double sum = 0.0;
    for (int64_t s = 0; s < S; ++s) sum += value_out[s];
    *mean_out = S > 0 ? sum / (double)S : 0.0;
  }
  return 0;
}

/* Reinsertion with route options (Sec. 2 Instantiation B: an entry of the
 * transition matrix may itself be a minimum over candidate route options,
 * A(I,J) = min_r A(I,J;r)).  Reading: on day t the delivery q = U - I can
 * ride any route r in 0..K-1 whose residual capacity cap[s][t][r] is at least
 * q, at insertion cost rcost[t][r] + unit_cost * q; no route, no delivery.
 *   nd(I)   = e(I - d_t) + C_{t+1}(max(0, I - d_t))
 *   dv_r(I) = rcost[t][r] + unit_cost (U-I) + e(U - d_t) + C_{t+1}(max(0, U - d_t))
 *   C_t(I)  = min(nd, min over feasible r of dv_r), I < U (I = U: nd only)
 * Decision: 0 = no delivery, r + 1 = route r; ties keep no delivery, then the
 * smallest r.  marg = gap between the best and the second-best action over
 * max(|best|, |second|) (+inf with a single action). */
static double reinsert_routes_one(const inv_t* m, int K, const float* rcost,
                                  const int32_t* cap, int I0, const int32_t* d, double* C,
                                  uint8_t* dec, double* marg, uint8_t* policy,
                                  double* value0) {
  const int T = m->T, U = m->U, W = U + 1;
  for (int I = 0; I < W; ++I) C[(size_t)T * W + I] = 0.0;
  for (int t = T - 1; t >= 0; --t) {
    const int64_t dt = d[t];
    const double* Cn = C + (size_t)(t + 1) * W;
    double* Ct = C + (size_t)t * W;
    for (int I = 0; I < W; ++I) {
      const int64_t x0 = (int64_t)I - dt;
      const double nd = end_cost(m, x0) + Cn[x0 > 0 ? x0 : 0];
      double best = nd, second = INFINITY;
      uint8_t a = 0;
      if (I < U) {
        const int q = U - I;
        const int64_t x1 = (int64_t)U - dt;
        const double e1 = end_cost(m, x1), c1 = Cn[x1 > 0 ? x1 : 0];
        for (int r = 0; r < K; ++r) {
          if (cap[(size_t)t * K + r] < q) continue;
          /* summed in the order of the two-action DP: F(q) + e + C */
          const double dv = ((double)rcost[(size_t)t * K + r] + m->unit_cost * (double)q) + e1 + c1;
          if (dv < best) {
            second = best;
            best = dv;
            a = (uint8_t)(r + 1);
          } else if (dv < second) {
            second = dv;
          }
        }
      }
      Ct[I] = best;
      dec[(size_t)t * W + I] = a;
      if (marg) {
        const double den = fmax(fabs(best), fabs(second));
        marg[(size_t)t * W + I] =
            isinf(second) ? INFINITY : (den > 0 ? (second - best) / den : 0.0);
      }
    }
  }
  if (value0)
    for (int I = 0; I < W; ++I) value0[I] = C[I];
  if (policy) {
    int64_t I = I0;
    for (int t = 0; t < T; ++t) {
      const uint8_t a = dec[(size_t)t * W + I];
      policy[t] = a;
      const int64_t x = (a ? U : I) - d[t];
      I = x > 0 ? x : 0;
    }
  }
  return C[I0];
}

/* Route-option reinsertion over S scenarios: rcost[T*K] shared, cap[S*T*K]
 * per scenario (cap[(s*T + t)*K + r]); other arguments as oracle_reinsert;
 * policy_out holds 0 (no delivery) or r + 1. */
int oracle_reinsert_routes(int T, int U, int I0, double h, double p, double unit_cost, int K,
                           const float* rcost, const int32_t* cap, const double* H,
                           int64_t S, const int32_t* cons, double* value_out,
                           uint8_t* policy_out, double* value0_out, double* margin_out,
                           double* mean_out, int nthreads) {
  if (T <= 0 || U < 0 || I0 < 0 || I0 > U || S < 0 || K < 0 || K > 254 || !value_out ||
      (K > 0 && (!rcost || !cap)))
    return -1;
  inv_t m = {T, U, h, p, unit_cost, NULL, H};
  const size_t W = (size_t)U + 1;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
#endif
  {
    double* C = (double*)malloc(sizeof(double) * (size_t)(T + 1) * W);
    uint8_t* dec = (uint8_t*)malloc((size_t)T * W);
    if (!C || !dec) bad = 1;
    else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
      for (int64_t s = 0; s < S; ++s) {
        value_out[s] = reinsert_routes_one(
            &m, K, rcost, cap + (size_t)s * T * K, I0, cons + s * T, C, dec,
            margin_out ? margin_out + (size_t)s * T * W : NULL,
            policy_out ? policy_out + s * T : NULL,
            value0_out ? value0_out + (size_t)s * W : NULL);
      }
    }
    free(C);
    free(dec);
  }
  if (bad) return -2;
  if (mean_out) {
    double sum = 0.0;
    for (int64_t s = 0; s < S; ++s) sum += value_out[s];
    *mean_out = S > 0 ? sum / (double)S : 0.0;
  }
  return 0;
}

/* Forward recursion of Eq. eqdp2 for one scenario: J_0 = one-hot at I0
 * (0 at I0, +inf elsewhere), and for each day t the transition matrix
 *   A_t(I,J) = min over q in {0, U-I} with max(0, I+q-d_t) = J of
 *              F_t(q) + e(I+q-d_t),   +inf if no such q,
 * is built explicitly (A_out, optional, [T*(U+1)*(U+1)]) and
 * J_{t+1} = A_t^T (min,+) J_t is taken with oracle_minplus_matvec.
 * Jhist_out (optional) [(T+1)*(U+1)] receives J_0..J_T.  Returns
 * min_J J_T(J), which must equal the backward value C_0(I0). */
double oracle_reinsert_forward(int T, int U, int I0, double h, double p,
                               double unit_cost, const float* fixed,
                               const double* H, const int32_t* cons,
                               double* A_out, double* Jhist_out) {
  inv_t m = {T, U, h, p, unit_cost, fixed, H};
  const int W = U + 1;
  double* A = (double*)malloc(sizeof(double) * (size_t)W * W);
  double* J = (double*)malloc(sizeof(double) * (size_t)W);
  double* Jn = (double*)malloc(sizeof(double) * (size_t)W);
  if (!A || !J || !Jn) { free(A); free(J); free(Jn); return NAN; }
  for (int I = 0; I < W; ++I) J[I] = (I == I0) ? 0.0 : INFINITY;
  if (Jhist_out) memcpy(Jhist_out, J, sizeof(double) * (size_t)W);
  for (int t = 0; t < T; ++t) {
    const int64_t dt = cons[t];
    for (size_t e = 0; e < (size_t)W * W; ++e) A[e] = INFINITY;
    for (int I = 0; I < W; ++I) {
      int nq = (I < U) ? 2 : 1; /* at I = U both actions are q = 0 (R2) */
      for (int k = 0; k < nq; ++k) {
        int q = k == 0 ? 0 : U - I;
        int64_t x = (int64_t)I + q - dt;
        int Jx = (int)(x > 0 ? x : 0);
        double c = route_cost(&m, t, q) + end_cost(&m, x);
        double* a = &A[(size_t)I * W + Jx];
        if (c < *a) *a = c;
      }
    }
    if (A_out) memcpy(A_out + (size_t)t * W * W, A, sizeof(double) * (size_t)W * W);
    oracle_minplus_matvec(W, W, A, J, Jn, NULL);
    memcpy(J, Jn, sizeof(double) * (size_t)W);
    if (Jhist_out) memcpy(Jhist_out + (size_t)(t + 1) * W, J, sizeof(double) * (size_t)W);
  }
  double best = INFINITY;
  for (int I = 0; I < W; ++I) best = J[I] < best ? J[I] : best;
  free(A); free(J); free(Jn);
  return best;
}
